// Internal context and graph objects (runtime.cu, tuner.cu).
#pragma once
#include <list>
#include <map>
#include <memory>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <vector>

#include "host_pool.h"
#include "internal.h"
#include "batch_kernels.cuh"
#include "kernels.cuh"
#include "bulk_config.h"

namespace mpt {

constexpr uint32_t kMaxStageSlots = 4;
constexpr uint32_t kLaneStreams = 4;  // streams per eager lane: copy-engine chains (two for staged hops)

struct GraphKey {
  uint64_t src, dst, nbytes, dir, plan_hash;
  bool operator==(const GraphKey& o) const {
    return src == o.src && dst == o.dst && nbytes == o.nbytes && dir == o.dir && plan_hash == o.plan_hash;
  }
};
struct GraphKeyHash {
  size_t operator()(const GraphKey& k) const { return (size_t)fnv1a(&k, sizeof k); }
};

// Per-path lane of the eager engine: hop-one and hop-two streams, per-slot events of the
// two-slot staging ring, and the lane's staging buffers (grown on demand).
struct EagerLane {
  cudaStream_t s[kLaneStreams] = {};
  cudaEvent_t join[kLaneStreams] = {};         // end of each extra copy-engine chain of a launch
  cudaEvent_t hop1[kMaxStageSlots] = {};
  cudaEvent_t hop2[kMaxStageSlots] = {};
  unsigned long long hop2_capture[kMaxStageSlots] = {};  // capture id the hop2 event was recorded in (0 = none)
  cudaEvent_t done = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;      // lane timers (MPT_TRACE_LANES)
  void* host_stage = nullptr;
  uint64_t host_stage_bytes = 0;
  void* dev_stage = nullptr;
  uint64_t dev_stage_bytes = 0;
};

// One tuned choice: the path set for a (direction, mode, log2 size bucket).
struct TuneEntry {
  uint32_t npaths = 0;
  uint32_t layout = 0;
  mpt_path_spec paths[4] = {};
  double us = 0;
};

// A registered arena: batch descriptors inside it skip per-pointer runtime queries.
struct Arena {
  uint64_t base, bytes;
  int kind;  // 0 device, 1 page-locked host
};

// One slot of the batch ring (see batch.cu).
struct BatchSlot {
  uint32_t max_xfers = 0;
  size_t table_bytes = 0, ctrl_bytes = 0;
  size_t desc_off = 0;          // descriptors' offset in the table (after header and lane map)
  uint8_t* h_table = nullptr;   // page-locked table, its used part copied to d_table by the graph
  uint32_t* h_flags = nullptr;  // page-locked, mapped: per-descriptor completion epochs
  unsigned long long* h_stamps = nullptr;  // page-locked, mapped: first and last CTA start
  void* d_mem = nullptr;
  uint8_t* d_table = nullptr;
  uint8_t* d_ctrl = nullptr;
  unsigned long long* d_times = nullptr;
  BatchArgs args{};
  cudaGraph_t graph[2] = {nullptr, nullptr};      // [0] k_batch, [1] k_batch_any
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaGraphNode_t table_cp[2] = {nullptr, nullptr};  // the table copy node of each graph
  size_t table_cp_bytes[2] = {0, 0};                 // and the size it copies now
  cudaEvent_t done_ev = nullptr;
  cudaEvent_t t0_ev = nullptr, t1_ev = nullptr;  // timing events around the replay (batch_timing)
  uint32_t epoch = 0;
  bool held = false;
  bool timed = false;  // the last replay was bracketed by t0_ev / t1_ev
  size_t n = 0;
  // DMA lanes: for each direction (D2D, H2D, D2H) `lanes` chains of `items` copy-engine
  // memcpy nodes, each followed by a completion kernel; item k = (dir * lanes + lane) *
  // items + position.  Per batch the used memcpy nodes are retargeted and enabled, the
  // others disabled (no cost when no entry is large).
  uint32_t dma_lanes = 0, dma_items = 0;
  uint32_t* h_dma_map = nullptr;  // in the page-locked table: item -> descriptor (~0 unused)
  std::vector<cudaGraphNode_t> dma_cp[2], dma_fin[2];
  std::vector<uint8_t> dma_on[2];
  void* h_scratch = nullptr;      // page-locked 64 bytes: instantiation-time operand of host lanes
};

mpt_status batch_setup(mpt_ctx_t c);
void batch_teardown(mpt_ctx_t c);

// The checks mpt_batch_submit applies to each transfer on its own (direction, NULL
// pointers, memory kinds against the direction).  *src_kind / *dst_kind: 0 device, 1
// page-locked host, 2 pageable host (-1 when not checked).  The cross-transfer checks
// (overlaps) are the batch's.
mpt_status batch_check_xfer(mpt_ctx_t c, const mpt_xfer& x, int* src_kind, int* dst_kind);

// Device time in ms between the timing events around a finished batch's replay (from the
// stream reaching the replay to its end), or -1 when the batch was not timed.
float batch_gpu_ms(mpt_batch_t b);

// Time between the first and the last CTA start of a finished batch's kernel (global timer):
// near the launch time when the whole grid became resident at once.
uint64_t batch_cta_spread_ns(mpt_batch_t b);

inline uint32_t tune_key(uint32_t dir, uint32_t mode, uint32_t bucket) { return (dir << 16) | (mode << 8) | bucket; }

uint32_t size_bucket(uint64_t nbytes);
mpt_model default_model(uint32_t dir, uint32_t mode);

}  // namespace mpt

struct mpt_graph_s {
  int refs = 0;
  mpt_ctx_t ctx = nullptr;
  mpt::GraphKey key{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  mpt_graph_info info{};
  std::vector<void*> host_allocs, dev_allocs;
  uint64_t src_lo = 0, src_hi = 0, dst_lo = 0, dst_hi = 0;
  bool cached = false;
  std::list<mpt_graph_s*>::iterator lru_it;
  mpt_plan_s* eager_plan = nullptr;  // set when prepared for direct issue instead of a graph
  std::vector<std::unique_ptr<mpt::HostCopyJob>> host_jobs;  // userData of this graph's host nodes
};

struct mpt_ctx_s {
  int device = 0;
  int sms = 0;
  int engines = 0;
  bool pageable = false;              // the GPU reaches pageable host memory (coherent host)
  uint32_t* d_status = nullptr;       // device status word
  unsigned long long* d_hash = nullptr;
  uint64_t* d_wait_ns = nullptr;      // device word: wait limit of the staged consumer's flag waits
  mpt::EagerLane lane[MPT_MAX_PATHS];
  cudaEvent_t fork = nullptr;
  std::unordered_map<mpt::GraphKey, mpt_graph_s*, mpt::GraphKeyHash> cache;
  std::list<mpt_graph_s*> lru;        // front = most recently used
  std::unordered_set<mpt_graph_s*> live;  // every graph not yet released
  size_t cache_cap = 64;
  uint64_t stage_max = 8ull << 20;
  bool rebind_enabled = true;  // MPT_GRAPH_REBIND=0 turns the capture fast path off
  bool trace_lanes = false;    // time every lane of multi-path eager launches
  uint32_t traced = 0;         // lanes timed by the last such launch
  bool pdl = true;             // direct kernel issue overlaps the previous copy kernel's end
  uint32_t stage_slots = 3;    // pinned slots of the device-to-device host-staged path (MPT_STAGE_SLOTS)
  uint32_t bulk_cfg = 0;       // configuration of the bulk-copy kernel (MPT_BULK_CONFIG)
  uint32_t ce_lanes = 1;       // chains a copy-engine path's chunks are dealt over (MPT_CE_LANES)
  std::unique_ptr<mpt::HostCopyPool> host_pool;  // CPU hops of host-thread staging (made on first use)
  unsigned host_threads = 0;   // pool workers (MPT_HOST_THREADS; 0 = min(8, cores / 2) - 1)
  std::map<uint32_t, mpt::TuneEntry> tuned;  // tune_key -> choice
  // tuner scratch (grown on demand)
  void* tune_a = nullptr;
  void* tune_b = nullptr;
  uint64_t tune_dev_bytes = 0;
  void* tune_h = nullptr;
  uint64_t tune_host_bytes = 0;
  void* tune_pg = nullptr;            // pageable host buffer (MPT_MODE_PAGEABLE)
  void* tune_h2 = nullptr;            // page-locked host buffer of the opposite direction (MPT_MODE_DUPLEX)
  uint64_t tune_h2_bytes = 0;
  uint64_t tune_pg_bytes = 0;
  void* flush = nullptr;              // L2 flush buffer
  uint64_t flush_bytes = 0;
  // batched transfers
  std::vector<mpt::BatchSlot> slots;
  std::vector<mpt::Arena> arenas;
  uint32_t batch_slots = 0, batch_max_xfers = 0, batch_ctas = 0, batch_tile = 0;
  // mpt_batch_submit's per-batch scratch, kept to avoid allocating per batch
  std::vector<std::pair<uint64_t, uint64_t>> batch_spans;
  std::vector<uint32_t> batch_cand;
  std::vector<uint8_t> batch_to_dma;
  uint32_t batch_dma_lanes = 0, batch_dma_items = 0;  // per direction; items per lane
  uint64_t batch_dma_min = 0;                         // smallest entry a DMA lane takes
  bool batch_dma_set = false;                         // configured (else environment defaults)
  bool batch_timing = false;                          // bracket each batch replay with timing events
  bool batch_split = true;                            // link and device tiles claimed separately (MPT_BATCH_SPLIT)
  uint32_t batch_link_ctas = 0;                       // CTAs that may take link tiles (MPT_BATCH_LINK_CTAS; 0 = default)
  std::vector<cudaEvent_t> each_ev;                   // completion events of mpt_copy_each (grown on demand)
  std::unordered_map<uint64_t, uint64_t> host_bufs;   // page-locked buffers mpt_host_alloc made: address -> bytes
};
