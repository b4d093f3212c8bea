// Configurations of the bulk-copy SM kernel (copy_bulk.cu), shared by the runtime, the tuner
// and the argument builder.  Kept apart from kernels.cuh so that the other copy kernels'
// sources do not change with them.
#pragma once
#include <cstdint>

namespace mpt {

// One configuration: a ring of `stages` shared-memory stages of `stage_bytes` (one
// cp.async.bulk load and one store per tile), stores allowed to be still reading shared
// memory for `keep` tiles behind the newest, `ctas_per_sm` CTAs resident per SM, and the
// kernel instantiated for it.
struct BulkConfig {
  uint32_t stages;
  uint32_t stage_bytes;
  uint32_t keep;
  uint32_t ctas_per_sm;
  const void* fn;
};
uint32_t bulk_config_count();
const BulkConfig& bulk_config(uint32_t i);  // i < bulk_config_count(), else the default
constexpr uint32_t kBulkDefaultConfig = 3;

}  // namespace mpt
