// Internal interface between the runtime (graph builder, eager engine) and the CUDA
// kernels of the transfer paths.  Not part of the public ABI (include/mpt.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpt {

// ---- byte-range copies (SM copy kernel, zero-copy kernel) ------------------------

constexpr int kInlineRanges = 16;     // ranges carried by value in one launch
constexpr int kVecThreads = 512;      // vec128 kernel block size
constexpr int kVecUnroll = 8;         // 16-byte vectors in flight per thread per tile
constexpr uint64_t kVecTileVecs = (uint64_t)kVecThreads * kVecUnroll;  // 64 KiB tiles
constexpr int kBulkThreads = 64;      // bulk kernel block: a producer warp and a consumer warp

// One contiguous range to copy: src + src_off -> dst + dst_off, `bytes` long.
// head: bytes copied singly until the destination is 16-byte aligned; shift: the source
// address modulo 16 after the head -- 0 when source and destination agree modulo 16, else
// each 16-byte destination word is assembled from two aligned source words.
struct RangeDesc {
  uint64_t src_off;
  uint64_t dst_off;
  uint64_t bytes;
  uint32_t head;
  uint32_t shift;
};

struct CopyArgs {
  const uint8_t* src;
  uint8_t* dst;
  uint32_t any_shift;                    // some range has shift != 0: launch an *_any kernel
  uint32_t nranges;
  uint32_t ntiles;                       // sum of tiles over ranges
  uint32_t tile_start[kInlineRanges + 1];
  RangeDesc r[kInlineRanges];
  uint32_t* status;                      // device status word (bounded waits)
  uint32_t bulk_cfg;                     // bulk variant: index into the bulk configurations
  uint32_t piece;                        // bulk variant: tile bytes (that configuration's stage)
};

// Fill `a` for up to kInlineRanges ranges with the tiling of `variant` (0 vec128,
// 1 bulk in configuration bulk_cfg (bulk_config.h), 2 zero-copy, 3 vec128 with 8 KiB tiles).  Returns
// kArgsOk, kArgsNeedVec when a bulk launch must fall back to vec128 (source and destination
// differ modulo 16, which cp.async.bulk cannot copy), or kArgsTooLarge.
constexpr int kArgsOk = 0, kArgsNeedVec = 1, kArgsTooLarge = 2;
int make_copy_args(CopyArgs& a, const void* src, void* dst, const RangeDesc* ranges, int n,
                   int variant, uint32_t* status, uint32_t bulk_cfg);

// *_any variants also copy ranges whose source and destination differ modulo 16
// (RangeDesc.shift != 0); the plain ones are leaner and need every shift to be 0.
__global__ void k_sm_copy_vec(CopyArgs a);
__global__ void k_sm_copy_vec_any(CopyArgs a);
__global__ void k_sm_copy_vec8k(CopyArgs a);
__global__ void k_sm_copy_vec8k_any(CopyArgs a);
__global__ void k_zc_copy(CopyArgs a);
__global__ void k_zc_copy_any(CopyArgs a);

// ---- flag-chained stage consumer (host-to-device staged path) ----------------------
// The copy engine fills stage chunk k and a memset node then sets ready[k] = 1.  The
// consumer kernel waits (bounded) for ready[k] and copies the chunk from the stage to its
// destination, counting the chunk's tiles in done[k].  A memset node at the head of every
// replay zeroes ready[] and done[] before any other node of the path runs.
struct StageChunk {
  uint64_t dst_off;    // destination offset of the chunk
  uint64_t stage_off;  // its offset in the stage buffer
  uint64_t bytes;
};

struct StageArgs {
  const uint8_t* stage;
  uint8_t* dst;
  const StageChunk* chunks;  // device table, nchunks entries
  uint32_t* ready;           // nchunks flags
  uint32_t* done;            // nchunks tile counters
  uint32_t nchunks;
  uint32_t tiles_per_chunk;  // ceil(max chunk bytes / tile)
  uint32_t* status;
  uint64_t timeout_ns;       // wait limit per chunk flag when wait_ns is null
  const uint64_t* wait_ns;   // the context's wait-limit word (device memory), read at each wait
};

__global__ void k_stage_consume(StageArgs a);

// ---- digest (test utility) -------------------------------------------------------
__global__ void k_hash(const uint8_t* p, uint64_t n, unsigned long long* out);

// Status codes written by kernels: (site << 8) | MPT_ETIMEDOUT.
constexpr uint32_t kSiteBulkLoad = 1;
constexpr uint32_t kSiteStageFlag = 2;
constexpr uint32_t kSiteBatch = 3;
constexpr uint32_t kSiteBulkArgs = 4;  // a bulk kernel given a tile size other than its stage

constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;  // 2 s
constexpr uint64_t kMaxWaitLimitNs = 10000000000ull;   // 10 s

}  // namespace mpt
