// Internal declarations shared by the host-side translation units of the library.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "mpt.h"

namespace mpt {

// Thread-local error message behind mpt_last_error().
void set_error(const char* fmt, ...);
mpt_status fail(mpt_status st, const char* fmt, ...);

bool kind_allowed(uint32_t dir, uint32_t kind);

// Validate a request and build its chunk list, sorted by (path, chunk index).
// path_bytes receives b_p for every path.
mpt_status build_chunks(uint64_t nbytes, uint32_t dir, const mpt_path_spec* paths, uint32_t npaths,
                        uint32_t align, uint32_t layout, std::vector<mpt_chunk>& out,
                        uint64_t* path_bytes);

uint64_t model_time(const mpt_model& m, uint32_t dir, const uint32_t* kinds, const uint64_t* bytes, uint32_t n,
                    uint64_t chunk);
mpt_status model_optimize(const mpt_model& m, uint64_t nbytes, uint32_t dir, const uint32_t* kinds, uint32_t n,
                          uint32_t align, uint64_t* best_bytes, uint64_t* best_chunk, uint64_t* best_ps);

uint64_t fnv1a(const void* data, size_t n, uint64_t h = 1469598103934665603ull);

}  // namespace mpt

struct mpt_plan_s {
  uint64_t nbytes = 0;
  uint32_t dir = 0, align = 16, layout = 0, npaths = 0;
  mpt_path_spec paths[MPT_MAX_PATHS] = {};
  uint64_t path_bytes[MPT_MAX_PATHS] = {};
  std::vector<mpt_chunk> chunks;  // sorted by (path_index, chunk_index)
  uint32_t first_chunk[MPT_MAX_PATHS + 1] = {};  // chunks of path p: [first[p], first[p+1])
  uint64_t hash = 0;
};
