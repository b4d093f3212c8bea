// Interface of the batched-transfer kernels (persistent descriptor-table kernel and the
// completion kernel of its copy-engine lanes) between batch.cu and the runtime.  Kept apart
// from kernels.cuh, which the copy kernels are compiled from.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mpt {

// ---- batched transfers: persistent descriptor-table kernel --------------------------
constexpr uint32_t kDescHostDst = 1;   // destination is host memory: publish with system fences
constexpr uint32_t kDescHostSide = 2;  // one side is host memory: coherent loads, no read-only path
constexpr uint32_t kDescDma = 4;       // moved by a copy-engine lane, not by the kernel (ntiles 0)

// Tiles come in two classes, each numbered from 0 and claimed through its own cursor: link
// tiles (one side in host memory: they move over the host link) and device tiles (both sides
// in this GPU's memory).  CTAs [0, link_ctas) claim link tiles first and move to device
// tiles when those run out; the others claim device tiles only.  The link, which bounds a
// mixed batch, stays busy from the start while the device tiles run beside it, and no more
// of its traffic is in flight than the link group keeps there.
struct BatchHeader {
  uint32_t n;            // descriptors in this batch
  uint32_t total_tiles;  // sum of tiles over descriptors, both classes
  uint32_t tile_bytes;
  uint32_t epoch;        // value written to a finished descriptor's host flag
  uint32_t link_tiles;   // tiles of the link class (the rest are device tiles)
  uint32_t n_link;       // descriptors with tiles in the link class: order[0, n_link)
  uint32_t n_tiled;      // descriptors with tiles: order[n_link, n_tiled) are the device class
  uint32_t link_ctas;    // CTAs that may take link tiles (the first ones of the grid)
};

struct BatchDesc {
  uint64_t src, dst, bytes;
  uint32_t first_tile;  // prefix sum of tiles before this descriptor, within its class
  uint32_t ntiles;      // max(1, ceil(bytes / tile)); 0 for a descriptor a DMA lane moves
  uint32_t flags;
  uint32_t pad;
};

// Device table of one batch, packed so that a batch of n descriptors is one copy of its
// first bytes: header | DMA-lane map | desc[n] | order[n], where order lists the
// descriptors with tiles, link class first (its address follows from n).
//
// The launch counters (cursors, per-descriptor tile counts, started and exited CTAs, the
// start time) are zero when a launch begins and the kernel leaves them zero: the CTA that
// counts a descriptor's last tile clears that descriptor's count, and the last CTA to exit,
// once no CTA can claim any more, clears the rest.  No reset node runs between launches.
struct BatchArgs {
  const BatchHeader* hdr;
  const BatchDesc* desc;         // desc[0..n); order[0..n) follows it
  uint32_t* cursor;              // next link tile to claim
  uint32_t* cursor_dev;          // next device tile to claim
  unsigned long long* start_inv; // ~(kernel start time), max over CTAs, during a launch
  unsigned long long* start_out; // the launch's ~(start time), kept after the launch
  uint32_t* done;                // tiles finished per descriptor
  unsigned long long* times;     // completion time per descriptor (global timer, ns)
  uint32_t* host_flags;          // device alias of page-locked flags, one per descriptor
  uint32_t* started;             // CTAs that have started
  uint32_t* exited;              // CTAs that have stopped claiming
  unsigned long long* host_stamps;  // device alias of page-locked [first, last] CTA start times
};

// Completion of one DMA-lane item: dma_map[item] is the descriptor its copy-engine node
// moved (~0 when the item is unused); stamps its time and raises its host flag.
__global__ void k_batch_dma_done(BatchArgs a, const uint32_t* dma_map, uint32_t item);

// k_batch needs every descriptor's source and destination to agree modulo 16;
// k_batch_any copies any alignment.
__global__ void k_batch(BatchArgs a);
__global__ void k_batch_any(BatchArgs a);

}  // namespace mpt
