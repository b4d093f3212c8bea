// Runtime of the multi-path transfer library: contexts, the CUDA graph engine and its
// LRU cache (Sec. 4.2), graph construction per path kind (Algorithms 1 and 2), the eager
// runtime pipelining engine (Sec. 4.3), and the C ABI entry points of mpt.h that need
// the GPU.
#include <dlfcn.h>

#include <algorithm>
#include <cctype>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <list>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "ctx.h"

namespace mpt {
const char* last_error_cstr();
}

#define CUDA_TRY(expr)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return mpt::fail(MPT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

namespace mpt {
namespace {

double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

uint64_t env_u64(const char* name, uint64_t dflt) {
  const char* v = std::getenv(name);
  if (!v || !*v) return dflt;
  char* end = nullptr;
  unsigned long long x = std::strtoull(v, &end, 0);
  return (end && *end == 0) ? (uint64_t)x : dflt;
}

enum MemKind { kMemDevice, kMemHost, kMemPageable, kMemOther };

// kMemPageable: ordinary (not page-locked) host memory, which the GPU reaches directly
// only when the device reports pageableMemoryAccess (coherent Grace hosts).
MemKind classify(const void* p, int device, bool pageable_ok = false) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return kMemOther;
  }
  if ((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device)
    return kMemDevice;
  if (a.type == cudaMemoryTypeHost) return kMemHost;
  if (a.type == cudaMemoryTypeUnregistered && p && pageable_ok) return kMemPageable;
  return kMemOther;
}

constexpr uint32_t kDefaultConsumerCtas = 32;

}  // namespace
}  // namespace mpt

namespace mpt {
namespace {

void graph_destroy_exec(mpt_graph_s* g) {
  delete g->eager_plan;
  g->eager_plan = nullptr;
  // A launch still in flight may not have run its host nodes yet: their jobs must outlive it.
  if (!g->host_jobs.empty()) cudaDeviceSynchronize();
  g->host_jobs.clear();
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  g->exec = nullptr;
  g->graph = nullptr;
  for (void* p : g->dev_allocs) cudaFree(p);
  for (void* p : g->host_allocs) cudaFreeHost(p);
  g->dev_allocs.clear();
  g->host_allocs.clear();
}

void graph_unref(mpt_graph_s* g) {
  if (--g->refs > 0) return;
  if (g->ctx) g->ctx->live.erase(g);
  graph_destroy_exec(g);
  delete g;
}

void cache_drop(mpt_ctx_t c, mpt_graph_s* g) {
  c->cache.erase(g->key);
  c->lru.erase(g->lru_it);
  g->cached = false;
  graph_unref(g);
}

// Default grids, from measurements on GB300 (CUDA events, back-to-back launches of one
// message): both SM copy kernels want many waves of CTAs, so that the block scheduler evens
// out SMs that stream at different rates.  With one wave every SM gets the same number of
// tiles and the faster ones idle (bulk kernel, one CTA per SM: 12 % of the elapsed cycles,
// 6.40 TB/s at 1 GiB).  The vec128 kernel: 64 CTAs per SM (a 64 KiB tile or two each at
// 1 GiB), 6.98 TB/s at 1 GiB against 6.80 with 16 per SM; the bulk kernel: 32 CTAs per SM,
// 6.99-7.02 TB/s at 1-4 GiB.  The zero-copy kernel saturates the host link with one CTA per SM.
uint32_t default_ctas(mpt_ctx_t c, uint32_t kind, uint32_t variant) {
  if (kind == MPT_PATH_ZC) return (uint32_t)c->sms;
  return (variant == MPT_SM_BULK ? 32u : 64u) * (uint32_t)c->sms;
}

// Chunks of one path merged into maximal contiguous ranges (CONTIG plans give one).
std::vector<RangeDesc> path_ranges(const mpt_plan_s* plan, uint32_t p) {
  std::vector<RangeDesc> out;
  for (uint32_t i = plan->first_chunk[p]; i < plan->first_chunk[p + 1]; ++i) {
    const mpt_chunk& c = plan->chunks[i];
    if (!out.empty() && out.back().src_off + out.back().bytes == c.offset) {
      out.back().bytes += c.bytes;
    } else {
      out.push_back(RangeDesc{c.offset, c.offset, c.bytes, 0, 0});
    }
  }
  return out;
}

void* kernel_fn(int variant, bool any_shift, uint32_t bulk_cfg) {
  if (variant == 1) return const_cast<void*>(bulk_config(bulk_cfg).fn);
  if (variant == 2) return any_shift ? reinterpret_cast<void*>(&k_zc_copy_any) : reinterpret_cast<void*>(&k_zc_copy);
  if (variant == 3)
    return any_shift ? reinterpret_cast<void*>(&k_sm_copy_vec8k_any) : reinterpret_cast<void*>(&k_sm_copy_vec8k);
  return any_shift ? reinterpret_cast<void*>(&k_sm_copy_vec_any) : reinterpret_cast<void*>(&k_sm_copy_vec);
}

// Build CopyArgs for up to kInlineRanges ranges; the bulk variant falls back to vec128
// when a range's source and destination differ modulo 16.
mpt_status prepare_copy(CopyArgs& a, int& variant, const void* src, void* dst, const RangeDesc* r, int n,
                        uint32_t* status, uint32_t bulk_cfg = kBulkDefaultConfig) {
  int rc = make_copy_args(a, src, dst, r, n, variant, status, bulk_cfg);
  if (rc == kArgsNeedVec) {
    variant = 0;
    rc = make_copy_args(a, src, dst, r, n, variant, status, bulk_cfg);
  }
  if (rc != kArgsOk) return fail(MPT_EINVAL, "copy of more than 2^31 tiles");
  return MPT_OK;
}

dim3 grid_for(const CopyArgs& a, uint32_t ctas) {
  return dim3(std::max<uint32_t>(1u, std::min<uint32_t>(ctas, a.ntiles)));
}

uint32_t block_for(int variant) { return variant == 1 ? (uint32_t)kBulkThreads : (uint32_t)kVecThreads; }
size_t smem_for(int variant, const CopyArgs& a) {
  if (variant != 1) return 0;
  const BulkConfig& b = bulk_config(a.bulk_cfg);
  return (size_t)b.stages * b.stage_bytes;
}

mpt_status add_copy_node(cudaGraph_t g, const cudaGraphNode_t* deps, size_t ndeps, cudaGraphNode_t* node,
                         int variant, const CopyArgs& a, uint32_t ctas, mpt_graph_info& info) {
  CopyArgs args = a;
  void* params[] = {&args};
  cudaKernelNodeParams kp{};
  kp.func = kernel_fn(variant, a.any_shift != 0, a.bulk_cfg);
  kp.gridDim = grid_for(a, ctas);
  kp.blockDim = dim3(block_for(variant));
  kp.sharedMemBytes = (unsigned)smem_for(variant, a);
  kp.kernelParams = params;
  CUDA_TRY(cudaGraphAddKernelNode(node, g, deps, ndeps, &kp));
  info.kernel_nodes++;
  return MPT_OK;
}

// `pdl`: launch with programmatic stream serialization, so that the kernel's launch overlaps
// the end of a copy kernel before it on the stream (the kernels wait for that kernel's
// completion before touching memory).  Not used inside a stream capture.
mpt_status launch_copy(cudaStream_t s, int variant, const CopyArgs& a, uint32_t ctas, bool pdl = false) {
  void* kfn = kernel_fn(variant, a.any_shift != 0, a.bulk_cfg);
  CopyArgs args = a;
  void* params[] = {&args};
  if (!pdl) {
    CUDA_TRY(cudaLaunchKernel(kfn, grid_for(a, ctas), dim3(block_for(variant)), params, smem_for(variant, a), s));
    return MPT_OK;
  }
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid_for(a, ctas);
  cfg.blockDim = dim3(block_for(variant));
  cfg.dynamicSmemBytes = smem_for(variant, a);
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_TRY(cudaLaunchKernelExC(&cfg, kfn, params));
  return MPT_OK;
}

// Kernel lane of a plan: every range of path p, 16 per launch / node.
template <typename Emit>
mpt_status for_each_copy(mpt_ctx_t c, const mpt_plan_s* plan, uint32_t p, const void* src, void* dst,
                         Emit emit) {
  const mpt_path_spec& spec = plan->paths[p];
  std::vector<RangeDesc> ranges = path_ranges(plan, p);
  int base_variant = spec.kind == MPT_PATH_ZC ? 2 : (spec.flags & MPT_SM_BULK ? 1 : (spec.flags & MPT_SM_TILE8K ? 3 : 0));
  for (size_t i = 0; i < ranges.size(); i += kInlineRanges) {
    int n = (int)std::min<size_t>(kInlineRanges, ranges.size() - i);
    int variant = base_variant;
    CopyArgs a;
    mpt_status st = prepare_copy(a, variant, src, dst, ranges.data() + i, n, c->d_status, c->bulk_cfg);
    if (st != MPT_OK) return st;
    if (a.ntiles == 0) continue;
    uint32_t ctas = spec.ctas ? spec.ctas : default_ctas(c, spec.kind, (uint32_t)variant);
    st = emit(variant, a, ctas);
    if (st != MPT_OK) return st;
  }
  return MPT_OK;
}

// The context's host copy pool, made on first use: MPT_HOST_THREADS workers, or one fewer
// than min(8, half the host cores) -- the thread running the host function copies a part
// too.  On a 16-core Grace host 7 workers move the most (72 GB/s at 8 MiB chunks); 15
// oversubscribe the cores the CUDA driver and the caller also use.
HostCopyPool* host_pool(mpt_ctx_t c) {
  if (!c->host_pool) {
    unsigned w = c->host_threads;
    if (w == 0) {
      const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
      w = std::min(8u, std::max(2u, hw / 2)) - 1;
    }
    try {
      c->host_pool.reset(new HostCopyPool(w));
    } catch (...) {
      return nullptr;
    }
  }
  return c->host_pool.get();
}

bool host_threads_path(const mpt_path_spec& s) { return s.kind == MPT_PATH_HS && (s.flags & MPT_HS_HOST_THREADS); }

bool has_host_threads(const mpt_plan_s* plan) {
  for (uint32_t p = 0; p < plan->npaths; ++p)
    if (plan->first_chunk[p + 1] > plan->first_chunk[p] && host_threads_path(plan->paths[p])) return true;
  return false;
}

mpt_status add_host_copy_node(mpt_graph_s* g, HostCopyPool* pool, const cudaGraphNode_t* dep, void* dst,
                              const void* src, size_t bytes, cudaGraphNode_t* node) {
  g->host_jobs.emplace_back(new HostCopyJob{pool, dst, src, bytes, false});
  cudaHostNodeParams hp{};
  hp.fn = host_copy_fn;
  hp.userData = g->host_jobs.back().get();
  CUDA_TRY(cudaGraphAddHostNode(node, g->graph, dep, dep ? 1 : 0, &hp));
  g->info.host_nodes++;
  return MPT_OK;
}

// ---- graph construction (Algorithm 1 CreateGraph, Algorithm 2 node helpers) ---------------

// Build the graph of `plan` for (dst, src) into g->graph and instantiate it (unless
// `instantiate` is false).  Staging buffers are allocated and owned by g, or, when `reuse`
// is given, taken in the same order from that graph (same plan => same buffers).
mpt_status build_graph(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, mpt_graph_s* g,
                       bool instantiate = true, const mpt_graph_s* reuse = nullptr) {
  mpt_graph_info& info = g->info;
  size_t host_i = 0, dev_i = 0;
  auto get_host = [&](size_t bytes, void** out) -> mpt_status {
    if (reuse) {
      if (host_i >= reuse->host_allocs.size()) return fail(MPT_EINVAL, "rebind: staging layout differs");
      *out = reuse->host_allocs[host_i++];
      return MPT_OK;
    }
    CUDA_TRY(cudaHostAlloc(out, bytes, cudaHostAllocPortable));
    g->host_allocs.push_back(*out);
    return MPT_OK;
  };
  auto get_dev = [&](size_t bytes, void** out) -> mpt_status {
    if (reuse) {
      if (dev_i >= reuse->dev_allocs.size()) return fail(MPT_EINVAL, "rebind: staging layout differs");
      *out = reuse->dev_allocs[dev_i++];
      return MPT_OK;
    }
    CUDA_TRY(cudaMalloc(out, bytes));
    g->dev_allocs.push_back(*out);
    return MPT_OK;
  };
  const double t0 = now_us();
  CUDA_TRY(cudaGraphCreate(&g->graph, 0));
  const double t1 = now_us();
  uint8_t* d8 = static_cast<uint8_t*>(dst);
  const uint8_t* s8 = static_cast<const uint8_t*>(src);

  for (uint32_t p = 0; p < plan->npaths; ++p) {
    const uint32_t lo = plan->first_chunk[p], hi = plan->first_chunk[p + 1];
    if (lo == hi) continue;
    const mpt_path_spec& spec = plan->paths[p];
    switch (spec.kind) {
      case MPT_PATH_CE: {
        // Algorithm 2 PeerToPeerCopy: one memcpy node per chunk.  The chunks are dealt round
        // robin over ce_lanes chains (one per copy engine by default), each chain a sequence
        // of nodes.  Measured on GB300 (64 MiB in 16 chunks): 32 us as three or four chains,
        // whether graph launches follow each other or not; as 16 independent branches, 34 us
        // alone but 63 us per launch when launches follow each other; as one chain, 50 us.
        const uint32_t lanes = std::max(1u, std::min(c->ce_lanes, hi - lo));
        std::vector<cudaGraphNode_t> tail(lanes, nullptr);
        for (uint32_t i = lo; i < hi; ++i) {
          const mpt_chunk& ch = plan->chunks[i];
          cudaGraphNode_t& prev = tail[(i - lo) % lanes];
          cudaGraphNode_t n;
          CUDA_TRY(cudaGraphAddMemcpyNode1D(&n, g->graph, prev ? &prev : nullptr, prev ? 1 : 0, d8 + ch.offset,
                                            s8 + ch.offset, ch.bytes, cudaMemcpyDefault));
          prev = n;
          info.memcpy_nodes++;
        }
        break;
      }
      case MPT_PATH_SM:
      case MPT_PATH_ZC: {
        mpt_status st = for_each_copy(c, plan, p, src, dst, [&](int variant, const CopyArgs& a, uint32_t ctas) {
          cudaGraphNode_t n;
          return add_copy_node(g->graph, nullptr, 0, &n, variant, a, ctas, info);
        });
        if (st != MPT_OK) return st;
        break;
      }
      case MPT_PATH_HS: {
        const uint64_t cb = spec.chunk_bytes;
        if (cb > c->stage_max)
          return fail(MPT_EINVAL, "mpt_capture: staged chunk %llu exceeds the stage size %llu (MPT_STAGE_BYTES)",
                      (unsigned long long)cb, (unsigned long long)c->stage_max);
        if (host_threads_path(spec)) {
          // Algorithm 2 StageHostCopy with a CPU hop: host buffer <-> pinned slot by the host
          // thread pool, slot <-> device by a copy engine; two slots, hop two of chunk k after
          // its hop one, hop one of chunk k+2 after hop two of chunk k.
          if (reuse) return fail(MPT_ENOTSUP, "rebind: host-thread staging is not retargeted in place");
          HostCopyPool* pool = host_pool(c);
          if (!pool) return fail(MPT_ENOMEM, "mpt_capture: host copy threads");
          void* stage = nullptr;
          mpt_status sa = get_host(2 * cb, &stage);
          if (sa != MPT_OK) return sa;
          info.staging_bytes += 2 * cb;
          uint8_t* st8 = static_cast<uint8_t*>(stage);
          cudaGraphNode_t prev_hop2[2] = {nullptr, nullptr};
          for (uint32_t i = lo; i < hi; ++i) {
            const mpt_chunk& ch = plan->chunks[i];
            const uint32_t slot = (i - lo) & 1u;
            uint8_t* sl = st8 + slot * cb;
            const cudaGraphNode_t* dep = prev_hop2[slot] ? &prev_hop2[slot] : nullptr;
            cudaGraphNode_t h1, h2;
            mpt_status st;
            if (plan->dir == MPT_H2D) {
              st = add_host_copy_node(g, pool, dep, sl, s8 + ch.offset, ch.bytes, &h1);
              if (st != MPT_OK) return st;
              CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2, g->graph, &h1, 1, d8 + ch.offset, sl, ch.bytes,
                                                cudaMemcpyHostToDevice));
            } else {
              CUDA_TRY(cudaGraphAddMemcpyNode1D(&h1, g->graph, dep, dep ? 1 : 0, sl, s8 + ch.offset, ch.bytes,
                                                cudaMemcpyDeviceToHost));
              st = add_host_copy_node(g, pool, &h1, d8 + ch.offset, sl, ch.bytes, &h2);
              if (st != MPT_OK) return st;
            }
            info.memcpy_nodes++;
            prev_hop2[slot] = h2;
          }
        } else if (plan->dir == MPT_D2D) {
          // Algorithm 2 StageHostCopy: device -> pinned host slot -> device; hop two of chunk k
          // after its hop one, hop one of chunk k+S after hop two of chunk k.  The paper double
          // buffers (S = 2); three slots keep both link directions busier (MPT_STAGE_SLOTS).
          // Hop ones also follow one another, and so do hop twos: one chain per link direction
          // (GB300, 512 MiB in 8 MiB chunks: 143-145 GB/s against 135-141 without those edges).
          void* stage = nullptr;
          const uint32_t S = c->stage_slots;
          mpt_status sa = get_host(S * cb, &stage);
          if (sa != MPT_OK) return sa;
          info.staging_bytes += S * cb;
          uint8_t* st8 = static_cast<uint8_t*>(stage);
          cudaGraphNode_t prev_hop2[kMaxStageSlots] = {};
          cudaGraphNode_t last1 = nullptr, last2 = nullptr;
          for (uint32_t i = lo; i < hi; ++i) {
            const mpt_chunk& ch = plan->chunks[i];
            const uint32_t slot = (i - lo) % S;
            cudaGraphNode_t h1, h2;
            std::vector<cudaGraphNode_t> d1, d2;
            if (prev_hop2[slot]) d1.push_back(prev_hop2[slot]);
            if (last1) d1.push_back(last1);
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&h1, g->graph, d1.empty() ? nullptr : d1.data(), d1.size(),
                                              st8 + slot * cb, s8 + ch.offset, ch.bytes, cudaMemcpyDeviceToHost));
            d2.push_back(h1);
            if (last2) d2.push_back(last2);
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2, g->graph, d2.data(), d2.size(), d8 + ch.offset, st8 + slot * cb,
                                              ch.bytes, cudaMemcpyHostToDevice));
            info.memcpy_nodes += 2;
            prev_hop2[slot] = h2;
            last1 = h1;
            last2 = h2;
          }
        } else if (plan->dir == MPT_H2D) {
          // Copy engine fills a device stage chunk by chunk; after each chunk a memset node
          // raises its ready flag; one consumer kernel moves chunks out as flags rise.  A
          // memset node at the head zeroes every flag and tile counter on each replay, and
          // all other nodes of the path run after it, so no flag left raised by an earlier
          // replay (one whose consumer gave up waiting) can be taken for this replay's.
          const uint32_t nch = hi - lo;
          std::vector<StageChunk> table(nch);
          uint64_t stage_bytes = 0;
          for (uint32_t k = 0; k < nch; ++k) {
            const mpt_chunk& ch = plan->chunks[lo + k];
            table[k] = StageChunk{ch.offset, stage_bytes, ch.bytes};
            stage_bytes += (ch.bytes + 255) & ~255ull;
          }
          void* dstage = nullptr;
          void* ctrl = nullptr;
          const size_t flags_bytes = (size_t)nch * 2 * sizeof(uint32_t);
          const size_t table_off = (flags_bytes + 255) & ~(size_t)255;
          mpt_status ga = get_dev(std::max<uint64_t>(stage_bytes, 256), &dstage);
          if (ga == MPT_OK) ga = get_dev(table_off + nch * sizeof(StageChunk), &ctrl);
          if (ga != MPT_OK) return ga;
          if (!reuse) {  // a reused control block already holds this table and resting flags
            CUDA_TRY(cudaMemset(ctrl, 0, flags_bytes));
            CUDA_TRY(cudaMemcpy(static_cast<uint8_t*>(ctrl) + table_off, table.data(), nch * sizeof(StageChunk),
                                cudaMemcpyHostToDevice));
          }
          info.staging_bytes += stage_bytes;
          uint32_t* ready = static_cast<uint32_t*>(ctrl);
          uint8_t* ds8 = static_cast<uint8_t*>(dstage);
          cudaGraphNode_t head;
          {
            cudaMemsetParams zp{};
            zp.dst = ctrl;
            zp.value = 0;
            zp.elementSize = 4;
            zp.width = 2 * nch;  // ready[nch] then done[nch]
            zp.height = 1;
            zp.pitch = 0;
            CUDA_TRY(cudaGraphAddMemsetNode(&head, g->graph, nullptr, 0, &zp));
            info.memset_nodes++;
          }
          // hop one of the chunks dealt over ce_lanes chains, as for a copy-engine path
          const uint32_t lanes = std::max(1u, std::min(c->ce_lanes, nch));
          std::vector<cudaGraphNode_t> tail(lanes, head);
          for (uint32_t k = 0; k < nch; ++k) {
            const mpt_chunk& ch = plan->chunks[lo + k];
            cudaGraphNode_t h1, m;
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&h1, g->graph, &tail[k % lanes], 1, ds8 + table[k].stage_off,
                                              s8 + ch.offset, ch.bytes, cudaMemcpyHostToDevice));
            info.memcpy_nodes++;
            // the flag's memset node sits in the chain, between this chunk's copy and the next
            // one of the lane: on GB300 (512 MiB in 8 MiB chunks) 192 GB/s, against 152-159
            // GB/s with the memset branching off the chain beside the next copy
            cudaMemsetParams mp{};
            mp.dst = ready + k;
            mp.value = 1;
            mp.elementSize = 4;
            mp.width = 1;
            mp.height = 1;
            mp.pitch = 0;
            CUDA_TRY(cudaGraphAddMemsetNode(&m, g->graph, &h1, 1, &mp));
            tail[k % lanes] = m;
            info.memset_nodes++;
          }
          StageArgs sa{};
          sa.stage = ds8;
          sa.dst = d8;
          sa.chunks = reinterpret_cast<const StageChunk*>(static_cast<uint8_t*>(ctrl) + table_off);
          sa.ready = ready;
          sa.done = ready + nch;
          sa.nchunks = nch;
          const uint64_t tile = kVecTileVecs * 16;
          sa.tiles_per_chunk = (uint32_t)((cb + tile - 1) / tile);
          sa.status = c->d_status;
          sa.timeout_ns = kDefaultTimeoutNs;
          sa.wait_ns = c->d_wait_ns;
          void* params[] = {&sa};
          cudaKernelNodeParams kp{};
          kp.func = reinterpret_cast<void*>(&k_stage_consume);
          const uint32_t ctas = spec.ctas ? spec.ctas : kDefaultConsumerCtas;
          kp.gridDim = dim3(std::min<uint32_t>(ctas, nch * sa.tiles_per_chunk));
          kp.blockDim = dim3(kVecThreads);
          kp.kernelParams = params;
          cudaGraphNode_t kn;
          CUDA_TRY(cudaGraphAddKernelNode(&kn, g->graph, &head, 1, &kp));
          info.kernel_nodes++;
        } else {
          // Device-to-host through a two-slot device stage: SM copy into the slot, then a
          // copy-engine hop to the host; a slot is refilled after its previous hop two.
          void* dstage = nullptr;
          mpt_status sa = get_dev(2 * cb, &dstage);
          if (sa != MPT_OK) return sa;
          info.staging_bytes += 2 * cb;
          uint8_t* ds8 = static_cast<uint8_t*>(dstage);
          cudaGraphNode_t prev_hop2[2] = {nullptr, nullptr};
          for (uint32_t i = lo; i < hi; ++i) {
            const mpt_chunk& ch = plan->chunks[i];
            const uint32_t slot = (i - lo) & 1u;
            RangeDesc r{ch.offset, slot * cb, ch.bytes, 0, 0};
            int variant = 0;
            CopyArgs a;
            mpt_status st = prepare_copy(a, variant, src, ds8, &r, 1, c->d_status);
            if (st != MPT_OK) return st;
            cudaGraphNode_t h1, h2;
            st = add_copy_node(g->graph, prev_hop2[slot] ? &prev_hop2[slot] : nullptr, prev_hop2[slot] ? 1 : 0, &h1,
                               variant, a, spec.ctas ? spec.ctas : default_ctas(c, MPT_PATH_SM, 0), info);
            if (st != MPT_OK) return st;
            CUDA_TRY(cudaGraphAddMemcpyNode1D(&h2, g->graph, &h1, 1, d8 + ch.offset, ds8 + slot * cb, ch.bytes,
                                              cudaMemcpyDeviceToHost));
            info.memcpy_nodes++;
            prev_hop2[slot] = h2;
          }
        }
        break;
      }
      default:
        return fail(MPT_EINVAL, "mpt_capture: unknown path kind %u", spec.kind);
    }
  }
  const double t2 = now_us();
  size_t nodes = 0;
  CUDA_TRY(cudaGraphGetNodes(g->graph, nullptr, &nodes));
  info.nodes = (uint32_t)nodes;
  if (nodes > 0 && instantiate) CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
  const double t3 = now_us();
  info.create_us = t1 - t0;
  info.construct_us = t2 - t1;
  info.instantiate_us = t3 - t2;
  return MPT_OK;
}

// True when [a, a+n) and [b, b+n) share a byte.
bool ranges_overlap(const void* a, const void* b, uint64_t n) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return n > 0 && (x < y ? y - x < n : x - y < n);
}

// Pointer kinds must fit the direction.  Host sides must be page-locked, except for plans
// whose paths all reach host memory without a copy engine touching it (pageable_ok).  The
// source and destination ranges must not overlap: the paths move disjoint chunks at the
// same time, so an overlapping copy would read bytes another path is writing.
mpt_status check_pointers(mpt_ctx_t c, uint32_t dir, const void* dst, const void* src, uint64_t nbytes,
                          bool pageable_ok = false) {
  if (ranges_overlap(dst, src, nbytes))
    return fail(MPT_EINVAL, "source %p and destination %p overlap within %llu bytes", src, dst,
                (unsigned long long)nbytes);
  const bool pg = pageable_ok;
  MemKind ks = classify(src, c->device, pg), kd = classify(dst, c->device, pg);
  if (ks == kMemPageable) ks = kMemHost;
  if (kd == kMemPageable) kd = kMemHost;
  const MemKind want_s = dir == MPT_H2D ? kMemHost : kMemDevice;
  const MemKind want_d = dir == MPT_D2H ? kMemHost : kMemDevice;
  if (ks != want_s)
    return fail(MPT_EINVAL, "source %p is not %s memory", src,
                want_s == kMemHost ? (pg ? "host" : "page-locked host (pageable memory needs a zero-copy-only plan)")
                                   : "device (this context's GPU)");
  if (kd != want_d)
    return fail(MPT_EINVAL, "destination %p is not %s memory", dst,
                want_d == kMemHost ? (pg ? "host" : "page-locked host (pageable memory needs a zero-copy-only plan)")
                                   : "device (this context's GPU)");
  return MPT_OK;
}

// Pageable host memory is allowed when every non-empty path of the plan is the zero-copy
// kernel (on devices that reach pageable memory: coherent hosts) or host-thread staging (CPU
// threads touch the host buffer; copy engines only the page-locked slots).
bool pageable_ok(mpt_ctx_t c, const mpt_plan_s* plan) {
  for (uint32_t p = 0; p < plan->npaths; ++p) {
    if (plan->first_chunk[p + 1] == plan->first_chunk[p]) continue;
    const mpt_path_spec& s = plan->paths[p];
    if (host_threads_path(s)) continue;
    if (s.kind == MPT_PATH_ZC && c->pageable) continue;
    return false;
  }
  return true;
}

// Retarget g at (dst, src) without instantiating: rebuild the node set for the new
// addresses (same plan, same staging buffers) and update the executable in place
// (cudaGraphExecUpdate).  ENOTSUP when the runtime cannot update (e.g. the kernel variant
// changes with the new alignment); g is then unchanged.
mpt_status rebind(mpt_ctx_t c, mpt_graph_s* g, const mpt_plan_s* plan, void* dst, const void* src) {
  const double t0 = now_us();
  // Host nodes carry their addresses in jobs that a launch in flight may still read.
  if (has_host_threads(plan)) return fail(MPT_ENOTSUP, "rebind: host-thread staging is not retargeted in place");
  if (!g->exec) {  // empty message: nothing to retarget
    g->info.update_us = now_us() - t0;
    g->info.rebinds++;
    return MPT_OK;
  }
  mpt_graph_s tmp;
  tmp.ctx = c;
  mpt_status st = build_graph(c, plan, dst, src, &tmp, false, g);
  if (st != MPT_OK) {
    if (tmp.graph) cudaGraphDestroy(tmp.graph);
    return st;
  }
  cudaGraphExecUpdateResultInfo ri{};
  const cudaError_t e = cudaGraphExecUpdate(g->exec, tmp.graph, &ri);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaGraphDestroy(tmp.graph);
    return fail(MPT_ENOTSUP, "rebind: the runtime cannot update this graph in place (%s)", cudaGetErrorString(e));
  }
  cudaGraphDestroy(g->graph);
  g->graph = tmp.graph;
  g->info.update_us = now_us() - t0;
  g->info.rebinds++;
  return MPT_OK;
}

void set_range(mpt_graph_s* g, uint64_t nbytes, const void* dst, const void* src) {
  g->src_lo = (uint64_t)(uintptr_t)src;
  g->src_hi = g->src_lo + nbytes;
  g->dst_lo = (uint64_t)(uintptr_t)dst;
  g->dst_hi = g->dst_lo + nbytes;
}

// ---- eager engine (Sec. 4.3 static runtime pipelining; Sec. 4.5 contention avoidance) ------

// Grow a lane's staging (never shrinks).  Earlier launches on the lane may still use the old
// buffer: the lane's streams are drained before it is freed.
mpt_status drain_lane(EagerLane& L) {
  for (cudaStream_t s : L.s)
    if (s) CUDA_TRY(cudaStreamSynchronize(s));
  return MPT_OK;
}

mpt_status grow_host(EagerLane& L, uint64_t bytes) {
  if (L.host_stage_bytes >= bytes) return MPT_OK;
  if (L.host_stage) {
    mpt_status st = drain_lane(L);
    if (st != MPT_OK) return st;
    CUDA_TRY(cudaFreeHost(L.host_stage));
  }
  L.host_stage = nullptr;
  L.host_stage_bytes = 0;
  CUDA_TRY(cudaHostAlloc(&L.host_stage, bytes, cudaHostAllocPortable));
  L.host_stage_bytes = bytes;
  return MPT_OK;
}

mpt_status grow_dev(EagerLane& L, uint64_t bytes) {
  if (L.dev_stage_bytes >= bytes) return MPT_OK;
  if (L.dev_stage) {
    mpt_status st = drain_lane(L);
    if (st != MPT_OK) return st;
    CUDA_TRY(cudaFree(L.dev_stage));
  }
  L.dev_stage = nullptr;
  L.dev_stage_bytes = 0;
  CUDA_TRY(cudaMalloc(&L.dev_stage, bytes));
  L.dev_stage_bytes = bytes;
  return MPT_OK;
}

mpt_status eager(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, cudaStream_t user) {
  if (plan->nbytes == 0) return MPT_OK;
  // One copy-engine or kernel path needs no fork and join: issue it on the caller's
  // stream directly (the cheapest launch for short messages).
  uint32_t nonempty = 0, only = 0;
  for (uint32_t p = 0; p < plan->npaths; ++p)
    if (plan->first_chunk[p + 1] > plan->first_chunk[p]) {
      nonempty++;
      only = p;
    }
  const bool ce_many = nonempty == 1 && plan->paths[only].kind == MPT_PATH_CE && c->ce_lanes > 1 &&
                       plan->first_chunk[only + 1] - plan->first_chunk[only] > 1;
  if (nonempty == 1 && plan->paths[only].kind != MPT_PATH_HS && !ce_many) {
    if (plan->paths[only].kind == MPT_PATH_CE) {
      for (uint32_t i = plan->first_chunk[only]; i < plan->first_chunk[only + 1]; ++i) {
        const mpt_chunk& ch = plan->chunks[i];
        CUDA_TRY(cudaMemcpyAsync(static_cast<uint8_t*>(dst) + ch.offset, static_cast<const uint8_t*>(src) + ch.offset,
                                 ch.bytes, cudaMemcpyDefault, user));
      }
      return MPT_OK;
    }
    bool pdl = c->pdl;
    if (pdl) {
      cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(user, &cap) != cudaSuccess) {
        cudaGetLastError();
        pdl = false;
      }
      if (cap != cudaStreamCaptureStatusNone) pdl = false;
    }
    return for_each_copy(c, plan, only, src, dst, [&](int variant, const CopyArgs& a, uint32_t ctas) {
      return launch_copy(user, variant, a, ctas, pdl);
    });
  }
  // A staged path allocates its staging on first use, which a stream capture forbids: refuse
  // before anything is issued, so the caller's capture stays intact.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  unsigned long long capture_id = 0;
  if (cudaStreamGetCaptureInfo(user, &cap, &capture_id) != cudaSuccess) {
    cudaGetLastError();
    cap = cudaStreamCaptureStatusNone;
  }
  if (cap != cudaStreamCaptureStatusActive) capture_id = 0;
  if (cap != cudaStreamCaptureStatusNone) {
    if (has_host_threads(plan))
      return fail(MPT_EINVAL, "mpt_launch_eager: host-thread staging cannot be captured from the eager engine "
                              "(each launch owns its CPU-hop jobs); build the graph with mpt_capture");
    for (uint32_t p = 0; p < plan->npaths; ++p) {
      if (plan->first_chunk[p + 1] == plan->first_chunk[p] || plan->paths[p].kind != MPT_PATH_HS) continue;
      const EagerLane& L = c->lane[p];
      const uint64_t have = plan->dir == MPT_D2D ? L.host_stage_bytes : L.dev_stage_bytes;
      const uint64_t slots = plan->dir == MPT_D2D ? c->stage_slots : 2u;
      if (have < slots * plan->paths[p].chunk_bytes)
        return fail(MPT_EINVAL, "mpt_launch_eager: the staged path allocates its staging on first use, which a "
                                "stream capture forbids; run the transfer once before capturing it");
    }
  }
  CUDA_TRY(cudaEventRecord(c->fork, user));
  c->traced = 0;
  uint8_t* d8 = static_cast<uint8_t*>(dst);
  const uint8_t* s8 = static_cast<const uint8_t*>(src);
  for (uint32_t p = 0; p < plan->npaths; ++p) {
    const uint32_t lo = plan->first_chunk[p], hi = plan->first_chunk[p + 1];
    if (lo == hi) continue;
    EagerLane& L = c->lane[p];
    const mpt_path_spec& spec = plan->paths[p];
    CUDA_TRY(cudaStreamWaitEvent(L.s[0], c->fork, 0));
    const bool trace = c->trace_lanes && capture_id == 0 && cap == cudaStreamCaptureStatusNone;
    if (trace) CUDA_TRY(cudaEventRecord(L.t0, L.s[0]));
    cudaStream_t last = L.s[0];
    switch (spec.kind) {
      case MPT_PATH_CE: {
        // chunks dealt round robin over the lane's streams, as the graph deals them over chains
        const uint32_t lanes = std::max(1u, std::min({c->ce_lanes, kLaneStreams, hi - lo}));
        for (uint32_t k = 1; k < lanes; ++k) CUDA_TRY(cudaStreamWaitEvent(L.s[k], c->fork, 0));
        for (uint32_t i = lo; i < hi; ++i) {
          const mpt_chunk& ch = plan->chunks[i];
          CUDA_TRY(cudaMemcpyAsync(d8 + ch.offset, s8 + ch.offset, ch.bytes, cudaMemcpyDefault, L.s[(i - lo) % lanes]));
        }
        for (uint32_t k = 1; k < lanes; ++k) {
          CUDA_TRY(cudaEventRecord(L.join[k], L.s[k]));
          CUDA_TRY(cudaStreamWaitEvent(L.s[0], L.join[k], 0));
        }
        break;
      }
      case MPT_PATH_SM:
      case MPT_PATH_ZC: {
        mpt_status st = for_each_copy(c, plan, p, src, dst, [&](int variant, const CopyArgs& a, uint32_t ctas) {
          return launch_copy(L.s[0], variant, a, ctas);
        });
        if (st != MPT_OK) return st;
        break;
      }
      case MPT_PATH_HS: {
        const uint64_t cb = spec.chunk_bytes;
        if (cb > c->stage_max)
          return fail(MPT_EINVAL, "mpt_launch_eager: staged chunk %llu exceeds the stage size %llu",
                      (unsigned long long)cb, (unsigned long long)c->stage_max);
        CUDA_TRY(cudaStreamWaitEvent(L.s[1], c->fork, 0));
        if (host_threads_path(spec)) {
          HostCopyPool* pool = host_pool(c);
          if (!pool) return fail(MPT_ENOMEM, "mpt_launch_eager: host copy threads");
          mpt_status st = grow_host(L, 2 * cb);
          if (st != MPT_OK) return st;
          uint8_t* stage = static_cast<uint8_t*>(L.host_stage);
          auto host_hop = [&](cudaStream_t s, void* to, const void* from, size_t n) -> mpt_status {
            HostCopyJob* job = new HostCopyJob{pool, to, from, n, true};
            const cudaError_t e = cudaLaunchHostFunc(s, host_copy_fn, job);
            if (e != cudaSuccess) {
              delete job;
              return fail(MPT_ECUDA, "cudaLaunchHostFunc: %s", cudaGetErrorString(e));
            }
            return MPT_OK;
          };
          for (uint32_t i = lo; i < hi; ++i) {
            const mpt_chunk& ch = plan->chunks[i];
            const uint32_t slot = (i - lo) & 1u;
            uint8_t* sl = stage + slot * cb;
            if (L.hop2_capture[slot] == capture_id) CUDA_TRY(cudaStreamWaitEvent(L.s[0], L.hop2[slot], 0));
            if (plan->dir == MPT_H2D) {
              st = host_hop(L.s[0], sl, s8 + ch.offset, ch.bytes);
              if (st != MPT_OK) return st;
            } else {
              CUDA_TRY(cudaMemcpyAsync(sl, s8 + ch.offset, ch.bytes, cudaMemcpyDeviceToHost, L.s[0]));
            }
            CUDA_TRY(cudaEventRecord(L.hop1[slot], L.s[0]));
            CUDA_TRY(cudaStreamWaitEvent(L.s[1], L.hop1[slot], 0));
            if (plan->dir == MPT_H2D) {
              CUDA_TRY(cudaMemcpyAsync(d8 + ch.offset, sl, ch.bytes, cudaMemcpyHostToDevice, L.s[1]));
            } else {
              st = host_hop(L.s[1], d8 + ch.offset, sl, ch.bytes);
              if (st != MPT_OK) return st;
            }
            CUDA_TRY(cudaEventRecord(L.hop2[slot], L.s[1]));
            L.hop2_capture[slot] = capture_id;
          }
          last = L.s[1];
          break;
        }
        uint8_t* stage;
        // device-to-device: the context's pinned slot count; host<->device: two device slots
        const uint32_t S = plan->dir == MPT_D2D ? c->stage_slots : 2u;
        if (plan->dir == MPT_D2D) {
          mpt_status st = grow_host(L, S * cb);
          if (st != MPT_OK) return st;
          stage = static_cast<uint8_t*>(L.host_stage);
        } else {
          mpt_status st = grow_dev(L, S * cb);
          if (st != MPT_OK) return st;
          stage = static_cast<uint8_t*>(L.dev_stage);
        }
        for (uint32_t i = lo; i < hi; ++i) {
          const mpt_chunk& ch = plan->chunks[i];
          const uint32_t slot = (i - lo) % S;
          uint8_t* sl = stage + slot * cb;
          // hop one may refill this slot only after the slot's previous hop two -- when that
          // hop two belongs to the same capture (or neither is captured): a capture cannot
          // wait on work recorded outside it
          if (L.hop2_capture[slot] == capture_id) CUDA_TRY(cudaStreamWaitEvent(L.s[0], L.hop2[slot], 0));
          if (plan->dir == MPT_D2H) {
            RangeDesc r{ch.offset, 0, ch.bytes, 0, 0};
            int variant = 0;
            CopyArgs a;
            mpt_status st = prepare_copy(a, variant, src, sl, &r, 1, c->d_status);
            if (st != MPT_OK) return st;
            st = launch_copy(L.s[0], variant, a, spec.ctas ? spec.ctas : default_ctas(c, MPT_PATH_SM, 0));
            if (st != MPT_OK) return st;
          } else {
            CUDA_TRY(cudaMemcpyAsync(sl, s8 + ch.offset, ch.bytes, cudaMemcpyDefault, L.s[0]));
          }
          CUDA_TRY(cudaEventRecord(L.hop1[slot], L.s[0]));
          CUDA_TRY(cudaStreamWaitEvent(L.s[1], L.hop1[slot], 0));
          if (plan->dir == MPT_H2D) {
            RangeDesc r{0, ch.offset, ch.bytes, 0, 0};
            int variant = 0;
            CopyArgs a;
            mpt_status st = prepare_copy(a, variant, sl, dst, &r, 1, c->d_status);
            if (st != MPT_OK) return st;
            st = launch_copy(L.s[1], variant, a, spec.ctas ? spec.ctas : default_ctas(c, MPT_PATH_SM, 0));
            if (st != MPT_OK) return st;
          } else {
            CUDA_TRY(cudaMemcpyAsync(d8 + ch.offset, sl, ch.bytes, cudaMemcpyDefault, L.s[1]));
          }
          CUDA_TRY(cudaEventRecord(L.hop2[slot], L.s[1]));
          L.hop2_capture[slot] = capture_id;
        }
        last = L.s[1];
        break;
      }
      default:
        return fail(MPT_EINVAL, "unknown path kind %u", spec.kind);
    }
    if (trace) {  // `last` ends after every hop of the lane
      CUDA_TRY(cudaEventRecord(L.t1, last));
      c->traced |= 1u << p;
    }
    CUDA_TRY(cudaEventRecord(L.done, last));
    CUDA_TRY(cudaStreamWaitEvent(user, L.done, 0));
  }
  return MPT_OK;
}

}  // namespace

mpt_status build_private_graph(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, mpt_graph_s* g) {
  g->ctx = c;
  mpt_status st = build_graph(c, plan, dst, src, g);
  if (st != MPT_OK) graph_destroy_exec(g);
  return st;
}

void free_private_graph(mpt_graph_s* g) { graph_destroy_exec(g); }

mpt_status run_eager(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, cudaStream_t s) {
  return eager(c, plan, dst, src, s);
}

}  // namespace mpt

using namespace mpt;

extern "C" {

const char* mpt_version(void) { return "mpt 0.1 (sm_103a)"; }

const char* mpt_last_error(void) { return last_error_cstr(); }

mpt_status mpt_ctx_create(int device, const char* tune_file, mpt_ctx_t* out) {
  if (!out) return fail(MPT_EINVAL, "mpt_ctx_create: out is NULL");
  *out = nullptr;
  int n = 0;
  CUDA_TRY(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) return fail(MPT_EINVAL, "mpt_ctx_create: device %d of %d", device, n);
  CUDA_TRY(cudaSetDevice(device));
  mpt_ctx_s* c = new mpt_ctx_s;
  c->device = device;
  auto bail = [&](mpt_status st) {
    mpt_ctx_destroy(c);
    return st;
  };
  int pageable = 0;
  if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->engines, cudaDevAttrAsyncEngineCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess)
    return bail(fail(MPT_ECUDA, "mpt_ctx_create: device attributes unavailable"));
  c->pageable = pageable != 0;
  void* words = nullptr;
  if (cudaMalloc(&words, 256) != cudaSuccess) return bail(fail(MPT_ENOMEM, "mpt_ctx_create: status word"));
  c->d_status = static_cast<uint32_t*>(words);
  c->d_hash = reinterpret_cast<unsigned long long*>(static_cast<uint8_t*>(words) + 128);
  c->d_wait_ns = reinterpret_cast<uint64_t*>(static_cast<uint8_t*>(words) + 64);
  if (cudaMemset(words, 0, 256) != cudaSuccess) return bail(fail(MPT_ECUDA, "mpt_ctx_create: memset"));
  {
    const uint64_t lim = kDefaultTimeoutNs;
    if (cudaMemcpy(c->d_wait_ns, &lim, sizeof lim, cudaMemcpyHostToDevice) != cudaSuccess)
      return bail(fail(MPT_ECUDA, "mpt_ctx_create: wait limit"));
  }
  for (uint32_t p = 0; p < MPT_MAX_PATHS; ++p) {
    EagerLane& L = c->lane[p];
    for (uint32_t i = 0; i < kLaneStreams; ++i)
      if (cudaStreamCreateWithFlags(&L.s[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&L.join[i], cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(MPT_ECUDA, "mpt_ctx_create: streams"));
    for (uint32_t i = 0; i < kMaxStageSlots; ++i)
      if (cudaEventCreateWithFlags(&L.hop1[i], cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&L.hop2[i], cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(MPT_ECUDA, "mpt_ctx_create: events"));
    if (cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&L.t0) != cudaSuccess || cudaEventCreate(&L.t1) != cudaSuccess)
      return bail(fail(MPT_ECUDA, "mpt_ctx_create: events"));
  }
  if (cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess)
    return bail(fail(MPT_ECUDA, "mpt_ctx_create: events"));
  for (uint32_t i = 0; i < bulk_config_count(); ++i) {
    const BulkConfig& b = bulk_config(i);
    if (cudaFuncSetAttribute(b.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(b.stages * b.stage_bytes)) !=
        cudaSuccess)
      return bail(fail(MPT_ECUDA, "mpt_ctx_create: bulk kernel shared memory"));
  }
  c->ce_lanes = (uint32_t)std::min<uint64_t>(16, std::max<uint64_t>(1, env_u64("MPT_CE_LANES", std::max(1, c->engines))));
  c->bulk_cfg = (uint32_t)env_u64("MPT_BULK_CONFIG", kBulkDefaultConfig);
  if (c->bulk_cfg >= bulk_config_count())
    return bail(fail(MPT_EINVAL, "mpt_ctx_create: MPT_BULK_CONFIG must be below %u", bulk_config_count()));
  c->cache_cap = (size_t)std::max<uint64_t>(1, env_u64("MPT_GRAPH_CACHE", 64));
  c->stage_max = std::max<uint64_t>(4096, env_u64("MPT_STAGE_BYTES", 8ull << 20));
  c->rebind_enabled = env_u64("MPT_GRAPH_REBIND", 1) != 0;
  c->trace_lanes = env_u64("MPT_TRACE_LANES", 0) != 0;
  c->pdl = env_u64("MPT_PDL", 1) != 0;
  c->stage_slots = (uint32_t)std::min<uint64_t>(kMaxStageSlots, std::max<uint64_t>(2, env_u64("MPT_STAGE_SLOTS", 3)));
  c->host_threads = (unsigned)std::min<uint64_t>(256, env_u64("MPT_HOST_THREADS", 0));
  const char* tf = tune_file && *tune_file ? tune_file : std::getenv("MPT_TUNE_FILE");
  if (tf && *tf) {
    mpt_status st = mpt_tune_load(c, tf);
    if (st != MPT_OK) return bail(st);
  } else if (env_u64("MPT_TUNE_DEFAULTS", 1) != 0) {
    // offline-tuned defaults for this device model, shipped next to the library as
    // tuned/<device name>.jsonl (Sec. 4.4: tuned values are the defaults)
    cudaDeviceProp prop;
    Dl_info info;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess &&
        dladdr(reinterpret_cast<void*>(&mpt_ctx_create), &info) && info.dli_fname) {
      std::string dir(info.dli_fname);
      dir = dir.substr(0, dir.find_last_of('/') + 1);
      std::string name(prop.name);
      for (char& ch : name)
        if (!std::isalnum((unsigned char)ch)) ch = '_';
      const std::string path = dir + "tuned/" + name + ".jsonl";
      if (FILE* f = std::fopen(path.c_str(), "r")) {
        std::fclose(f);
        mpt_status st = mpt_tune_load(c, path.c_str());
        if (st != MPT_OK) return bail(st);
      }
    }
  }
  *out = c;
  return MPT_OK;
}

mpt_status mpt_ctx_destroy(mpt_ctx_t c) {
  if (!c) return MPT_OK;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  batch_teardown(c);
  // Drop the cache's references; graphs the caller still holds lose their executable.
  while (!c->lru.empty()) cache_drop(c, c->lru.front());
  for (mpt_graph_s* g : c->live) {
    graph_destroy_exec(g);
    g->ctx = nullptr;
  }
  c->live.clear();
  for (uint32_t p = 0; p < MPT_MAX_PATHS; ++p) {
    EagerLane& L = c->lane[p];
    for (uint32_t i = 0; i < kLaneStreams; ++i) {
      if (L.s[i]) cudaStreamDestroy(L.s[i]);
      if (L.join[i]) cudaEventDestroy(L.join[i]);
    }
    for (uint32_t i = 0; i < kMaxStageSlots; ++i) {
      if (L.hop1[i]) cudaEventDestroy(L.hop1[i]);
      if (L.hop2[i]) cudaEventDestroy(L.hop2[i]);
    }
    if (L.done) cudaEventDestroy(L.done);
    if (L.t0) cudaEventDestroy(L.t0);
    if (L.t1) cudaEventDestroy(L.t1);
    if (L.host_stage) cudaFreeHost(L.host_stage);
    if (L.dev_stage) cudaFree(L.dev_stage);
  }
  if (c->fork) cudaEventDestroy(c->fork);
  if (c->d_status) cudaFree(c->d_status);
  if (c->tune_h2) cudaFreeHost(c->tune_h2);
  if (c->tune_a) cudaFree(c->tune_a);
  if (c->tune_b) cudaFree(c->tune_b);
  if (c->tune_h) cudaFreeHost(c->tune_h);
  std::free(c->tune_pg);
  if (c->flush) cudaFree(c->flush);
  delete c;
  return MPT_OK;
}

mpt_status mpt_ctx_info(mpt_ctx_t c, mpt_device_info* out) {
  if (!c || !out) return fail(MPT_EINVAL, "mpt_ctx_info: NULL argument");
  cudaDeviceProp prop;
  CUDA_TRY(cudaGetDeviceProperties(&prop, c->device));
  std::memset(out, 0, sizeof *out);
  std::snprintf(out->name, sizeof out->name, "%s", prop.name);
  out->device = c->device;
  out->sms = c->sms;
  out->copy_engines = c->engines;
  out->pageable_access = c->pageable ? 1 : 0;
  out->l2_bytes = (uint64_t)prop.l2CacheSize;
  out->memory_bytes = (uint64_t)prop.totalGlobalMem;
  return MPT_OK;
}

mpt_status mpt_trace_lanes(mpt_ctx_t c, uint32_t enable) {
  if (!c) return fail(MPT_EINVAL, "mpt_trace_lanes: NULL context");
  c->trace_lanes = enable != 0;
  c->traced = 0;
  return MPT_OK;
}

mpt_status mpt_lane_times(mpt_ctx_t c, float* out_ms, uint32_t cap, uint32_t* n) {
  if (!c || !n || (cap && !out_ms)) return fail(MPT_EINVAL, "mpt_lane_times: NULL argument");
  uint32_t k = 0;
  for (uint32_t p = 0; p < MPT_MAX_PATHS; ++p) {
    if (!(c->traced & (1u << p))) {
      if (p < cap) out_ms[p] = -1.0f;
      continue;
    }
    float ms = -1.0f;
    CUDA_TRY(cudaEventSynchronize(c->lane[p].t1));
    CUDA_TRY(cudaEventElapsedTime(&ms, c->lane[p].t0, c->lane[p].t1));
    if (p < cap) out_ms[p] = ms;
    k = p + 1;
  }
  *n = k;
  return MPT_OK;
}

mpt_status mpt_ctx_set_wait_limit(mpt_ctx_t c, uint64_t ns) {
  if (!c) return fail(MPT_EINVAL, "mpt_ctx_set_wait_limit: NULL context");
  if (ns > kMaxWaitLimitNs)
    return fail(MPT_EINVAL, "mpt_ctx_set_wait_limit: %llu ns exceeds the maximum of %llu ns", (unsigned long long)ns,
                (unsigned long long)kMaxWaitLimitNs);
  const uint64_t lim = ns ? ns : kDefaultTimeoutNs;
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(c->d_wait_ns, &lim, sizeof lim, cudaMemcpyHostToDevice));
  return MPT_OK;
}

mpt_status mpt_ctx_status(mpt_ctx_t c, uint32_t* site) {
  if (!c) return fail(MPT_EINVAL, "mpt_ctx_status: NULL context");
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaDeviceSynchronize());
  uint32_t w = 0;
  CUDA_TRY(cudaMemcpy(&w, c->d_status, sizeof w, cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(c->d_status, 0, sizeof w));
  if (site) *site = w >> 8;
  const uint32_t code = w & 0xffu;
  if (code == 0) return MPT_OK;
  return fail((mpt_status)code, "device wait gave up (site %u)", w >> 8);
}

mpt_status mpt_capture(mpt_ctx_t c, mpt_plan_t plan, void* dst, const void* src, mpt_graph_t* out) {
  if (!c || !plan || !out) return fail(MPT_EINVAL, "mpt_capture: NULL argument");
  *out = nullptr;
  CUDA_TRY(cudaSetDevice(c->device));
  if (plan->nbytes > 0) {
    mpt_status st = check_pointers(c, plan->dir, dst, src, plan->nbytes, pageable_ok(c, plan));
    if (st != MPT_OK) return st;
  }
  GraphKey key{(uint64_t)(uintptr_t)src, (uint64_t)(uintptr_t)dst, plan->nbytes, plan->dir, plan->hash};
  auto it = c->cache.find(key);
  if (it != c->cache.end()) {
    mpt_graph_s* g = it->second;
    c->lru.splice(c->lru.begin(), c->lru, g->lru_it);
    g->refs++;
    *out = g;
    return MPT_OK;
  }
  // An idle cached graph of the same plan (held by the cache alone) is retargeted in place
  // instead of instantiating a new one.
  if (c->rebind_enabled) {
    for (auto lit = c->lru.rbegin(); lit != c->lru.rend(); ++lit) {
      mpt_graph_s* g = *lit;
      if (g->refs != 1 || g->key.nbytes != key.nbytes || g->key.dir != key.dir || g->key.plan_hash != key.plan_hash)
        continue;
      if (rebind(c, g, plan, dst, src) != MPT_OK) break;
      c->cache.erase(g->key);
      g->key = key;
      set_range(g, plan->nbytes, dst, src);
      c->cache.emplace(key, g);
      c->lru.splice(c->lru.begin(), c->lru, g->lru_it);
      g->refs++;
      *out = g;
      return MPT_OK;
    }
  }
  mpt_graph_s* g = new mpt_graph_s;
  g->ctx = c;
  g->key = key;
  set_range(g, plan->nbytes, dst, src);
  mpt_status st = build_graph(c, plan, dst, src, g);
  if (st != MPT_OK) {
    graph_destroy_exec(g);
    delete g;
    return st;
  }
  while (c->cache.size() >= c->cache_cap && !c->lru.empty()) cache_drop(c, c->lru.back());
  g->refs = 2;  // the cache's and the caller's
  g->cached = true;
  c->lru.push_front(g);
  g->lru_it = c->lru.begin();
  c->cache.emplace(key, g);
  c->live.insert(g);
  *out = g;
  return MPT_OK;
}

mpt_status mpt_prepare(mpt_ctx_t c, mpt_plan_t plan, void* dst, const void* src, uint32_t mode, mpt_graph_t* out) {
  if (!c || !plan || !out) return fail(MPT_EINVAL, "mpt_prepare: NULL argument");
  if (mode > MPT_PREPARE_AUTO) return fail(MPT_EINVAL, "mpt_prepare: unknown mode %u", mode);
  *out = nullptr;
  if (mode == MPT_PREPARE_AUTO) {
    // graph or direct issue, whichever the tuner measured faster for this size bucket
    // (Sec. 4.4: tuned separately for graph and non-graph execution)
    const uint32_t b = size_bucket(plan->nbytes);
    auto g = c->tuned.find(tune_key(plan->dir, 0, b));
    auto e = c->tuned.find(tune_key(plan->dir, 1, b));
    mode = (g != c->tuned.end() && e != c->tuned.end() && e->second.us < g->second.us) ? MPT_PREPARE_EAGER
                                                                                       : MPT_PREPARE_GRAPH;
  }
  if (mode == MPT_PREPARE_GRAPH) return mpt_capture(c, plan, dst, src, out);
  CUDA_TRY(cudaSetDevice(c->device));
  if (plan->nbytes > 0) {
    mpt_status st = check_pointers(c, plan->dir, dst, src, plan->nbytes, pageable_ok(c, plan));
    if (st != MPT_OK) return st;
  }
  mpt_graph_s* g = new mpt_graph_s;
  g->ctx = c;
  g->key = GraphKey{(uint64_t)(uintptr_t)src, (uint64_t)(uintptr_t)dst, plan->nbytes, plan->dir, plan->hash};
  set_range(g, plan->nbytes, dst, src);
  g->eager_plan = new mpt_plan_s(*plan);
  g->info.mode = 1;
  g->refs = 1;
  c->live.insert(g);
  *out = g;
  return MPT_OK;
}

mpt_status mpt_launch(mpt_graph_t g, void* stream) {
  if (!g) return fail(MPT_EINVAL, "mpt_launch: NULL graph");
  if (!g->ctx) return fail(MPT_EINVAL, "mpt_launch: the graph's context was destroyed");
  if (g->eager_plan) {  // prepared for direct issue (mpt_prepare chose eager)
    CUDA_TRY(cudaSetDevice(g->ctx->device));
    return eager(g->ctx, g->eager_plan, reinterpret_cast<void*>(g->key.dst), reinterpret_cast<const void*>(g->key.src),
                 static_cast<cudaStream_t>(stream));
  }
  if (!g->exec) return MPT_OK;  // empty message: nothing to move
  CUDA_TRY(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
  return MPT_OK;
}

mpt_status mpt_graph_get_info(mpt_graph_t g, mpt_graph_info* out) {
  if (!g || !out) return fail(MPT_EINVAL, "mpt_graph_get_info: NULL argument");
  *out = g->info;
  return MPT_OK;
}

mpt_status mpt_graph_rebind(mpt_graph_t g, mpt_plan_t plan, void* dst, const void* src) {
  if (!g || !plan) return fail(MPT_EINVAL, "mpt_graph_rebind: NULL argument");
  mpt_ctx_t c = g->ctx;
  if (!c) return fail(MPT_EINVAL, "mpt_graph_rebind: the graph's context was destroyed");
  if (plan->hash != g->key.plan_hash || plan->nbytes != g->key.nbytes || plan->dir != g->key.dir)
    return fail(MPT_EINVAL, "mpt_graph_rebind: the plan is not the one the graph was captured from");
  CUDA_TRY(cudaSetDevice(c->device));
  if (plan->nbytes > 0) {
    mpt_status st = check_pointers(c, plan->dir, dst, src, plan->nbytes, pageable_ok(c, plan));
    if (st != MPT_OK) return st;
  }
  GraphKey key{(uint64_t)(uintptr_t)src, (uint64_t)(uintptr_t)dst, plan->nbytes, plan->dir, plan->hash};
  if (g->cached) {
    auto it = c->cache.find(key);
    if (it != c->cache.end() && it->second != g)
      return fail(MPT_EAGAIN, "mpt_graph_rebind: another cached graph already serves these addresses");
  }
  mpt_status st = rebind(c, g, plan, dst, src);
  if (st != MPT_OK) return st;
  if (g->cached) {
    c->cache.erase(g->key);
    c->cache.emplace(key, g);
  }
  g->key = key;
  set_range(g, plan->nbytes, dst, src);
  return MPT_OK;
}

mpt_status mpt_graph_release(mpt_graph_t g) {
  if (!g) return MPT_OK;
  graph_unref(g);
  return MPT_OK;
}

mpt_status mpt_graph_evict(mpt_ctx_t c, const void* ptr, uint32_t* n) {
  if (!c) return fail(MPT_EINVAL, "mpt_graph_evict: NULL context");
  const uint64_t a = (uint64_t)(uintptr_t)ptr;
  uint32_t dropped = 0;
  for (auto it = c->lru.begin(); it != c->lru.end();) {
    mpt_graph_s* g = *it++;
    const bool hit = (a >= g->src_lo && a < g->src_hi) || (a >= g->dst_lo && a < g->dst_hi) ||
                     (a == g->src_lo) || (a == g->dst_lo);
    if (hit) {
      cache_drop(c, g);
      dropped++;
    }
  }
  if (n) *n = dropped;
  return MPT_OK;
}

mpt_status mpt_launch_eager(mpt_ctx_t c, mpt_plan_t plan, void* dst, const void* src, void* stream) {
  if (!c || !plan) return fail(MPT_EINVAL, "mpt_launch_eager: NULL argument");
  CUDA_TRY(cudaSetDevice(c->device));
  if (plan->nbytes > 0) {
    mpt_status st = check_pointers(c, plan->dir, dst, src, plan->nbytes, pageable_ok(c, plan));
    if (st != MPT_OK) return st;
  }
  return eager(c, plan, dst, src, static_cast<cudaStream_t>(stream));
}

mpt_status mpt_sm_copy(mpt_ctx_t c, void* dst, const void* src, uint64_t nbytes, uint32_t variant, uint32_t ctas,
                       void* stream) {
  if (!c) return fail(MPT_EINVAL, "mpt_sm_copy: NULL context");
  if (variant > MPT_SM_TILE8K) return fail(MPT_EINVAL, "mpt_sm_copy: unknown variant %u", variant);
  if (nbytes == 0) return MPT_OK;
  if (!dst || !src) return fail(MPT_EINVAL, "mpt_sm_copy: NULL pointer");
  if (ranges_overlap(dst, src, nbytes)) return fail(MPT_EINVAL, "mpt_sm_copy: source and destination overlap");
  CUDA_TRY(cudaSetDevice(c->device));
  const MemKind ks = classify(src, c->device, c->pageable), kd = classify(dst, c->device, c->pageable);
  if (ks == kMemOther || kd == kMemOther)
    return fail(MPT_EINVAL, "mpt_sm_copy: pointers must be device or host memory the GPU can reach");
  const bool host = ks != kMemDevice || kd != kMemDevice;
  RangeDesc r{0, 0, nbytes, 0, 0};
  int v = host ? 2 : (variant == MPT_SM_TILE8K ? 3 : (int)variant);
  CopyArgs a;
  mpt_status st = prepare_copy(a, v, src, dst, &r, 1, c->d_status, c->bulk_cfg);
  if (st != MPT_OK) return st;
  const uint32_t g = ctas ? ctas : default_ctas(c, host ? MPT_PATH_ZC : MPT_PATH_SM, (uint32_t)v);
  return launch_copy(static_cast<cudaStream_t>(stream), v, a, g);
}

mpt_status mpt_hash_device(mpt_ctx_t c, const void* ptr, uint64_t nbytes, void* stream, uint64_t* out) {
  if (!c || !out) return fail(MPT_EINVAL, "mpt_hash_device: NULL argument");
  if (nbytes > 0 && !ptr) return fail(MPT_EINVAL, "mpt_hash_device: NULL pointer");
  CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CUDA_TRY(cudaMemsetAsync(c->d_hash, 0, sizeof(unsigned long long), s));
  const uint64_t words = (nbytes + 7) / 8;
  const uint32_t blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(4ull * c->sms, (words + 255) / 256));
  k_hash<<<blocks, 256, 0, s>>>(static_cast<const uint8_t*>(ptr), nbytes, c->d_hash);
  CUDA_TRY(cudaGetLastError());
  unsigned long long h = 0;
  CUDA_TRY(cudaMemcpyAsync(&h, c->d_hash, sizeof h, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  *out = h;
  return MPT_OK;
}

mpt_status mpt_selftest_flag_timeout(mpt_ctx_t c, uint64_t timeout_ns, uint32_t* site) {
  if (!c) return fail(MPT_EINVAL, "mpt_selftest_flag_timeout: NULL context");
  if (timeout_ns == 0 || timeout_ns > 10000000000ull)
    return fail(MPT_EINVAL, "mpt_selftest_flag_timeout: timeout must be in (0, 10 s]");
  CUDA_TRY(cudaSetDevice(c->device));
  CUDA_TRY(cudaDeviceSynchronize());
  // one staged chunk whose ready flag nothing ever raises
  void* mem = nullptr;
  CUDA_TRY(cudaMalloc(&mem, 8192));
  CUDA_TRY(cudaMemset(mem, 0, 8192));
  uint8_t* m8 = static_cast<uint8_t*>(mem);
  StageChunk ch{0, 0, 1024};
  CUDA_TRY(cudaMemcpy(m8 + 256, &ch, sizeof ch, cudaMemcpyHostToDevice));
  StageArgs sa{};
  sa.stage = m8 + 4096;
  sa.dst = m8 + 6144;
  sa.chunks = reinterpret_cast<const StageChunk*>(m8 + 256);
  sa.ready = reinterpret_cast<uint32_t*>(m8);
  sa.done = reinterpret_cast<uint32_t*>(m8 + 64);
  sa.nchunks = 1;
  sa.tiles_per_chunk = 1;
  sa.status = c->d_status;
  sa.timeout_ns = timeout_ns;
  k_stage_consume<<<1, kVecThreads>>>(sa);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(mem);
  if (e != cudaSuccess) return fail(MPT_ECUDA, "mpt_selftest_flag_timeout: %s", cudaGetErrorString(e));
  return mpt_ctx_status(c, site);
}

mpt_status mpt_host_alloc(mpt_ctx_t c, uint64_t nbytes, void** host, void** dev_alias) {
  if (!host) return fail(MPT_EINVAL, "mpt_host_alloc: host is NULL");
  *host = nullptr;
  if (dev_alias) *dev_alias = nullptr;
  if (c) CUDA_TRY(cudaSetDevice(c->device));
  if (cudaHostAlloc(host, std::max<uint64_t>(nbytes, 1), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    cudaGetLastError();
    *host = nullptr;
    return fail(MPT_ENOMEM, "mpt_host_alloc: %llu bytes", (unsigned long long)nbytes);
  }
  if (dev_alias && cudaHostGetDevicePointer(dev_alias, *host, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(*host);
    *host = nullptr;
    return fail(MPT_ECUDA, "mpt_host_alloc: no device address for the mapped buffer");
  }
  if (c) c->host_bufs[(uint64_t)(uintptr_t)*host] = nbytes;
  return MPT_OK;
}

mpt_status mpt_host_free(mpt_ctx_t c, void* p) {
  if (!p) return MPT_OK;
  if (c) {
    // cached graphs bound to the buffer must not outlive it: a graph whose memcpy nodes
    // refer to freed page-locked memory cannot be launched or retargeted safely
    auto it = c->host_bufs.find((uint64_t)(uintptr_t)p);
    if (it != c->host_bufs.end()) {
      const uint64_t a = it->first, b = it->first + std::max<uint64_t>(it->second, 1);
      for (auto lit = c->lru.begin(); lit != c->lru.end();) {
        mpt_graph_s* g = *lit++;
        const auto touches = [&](uint64_t lo, uint64_t hi) { return lo < b && a < std::max(hi, lo + 1); };
        if (touches(g->src_lo, g->src_hi) || touches(g->dst_lo, g->dst_hi)) cache_drop(c, g);
      }
      c->host_bufs.erase(it);
    }
  }
  CUDA_TRY(cudaFreeHost(p));
  return MPT_OK;
}

}  // extern "C"

