// mpt_plan and friends: the planning half of the C ABI.  Pure host code; runs without a
// GPU when every path carries an explicit chunk size.
#include <cstring>

#include "internal.h"

namespace mpt {
// Implemented by the runtime: fill chunk sizes (and, when whole_set, the path set and
// shares) from the context's tuner for this message size and direction.
mpt_status tuner_fill(mpt_ctx_t ctx, uint64_t nbytes, uint32_t dir, uint32_t mode, uint32_t align,
                      mpt_path_spec* specs, uint32_t* npaths, bool whole_set);
}  // namespace mpt

using namespace mpt;

extern "C" {

mpt_status mpt_plan(mpt_ctx_t ctx, uint64_t nbytes, uint32_t dir, const mpt_path_spec* paths, uint32_t npaths,
                    uint32_t align, uint32_t layout, mpt_plan_t* out) {
  if (!out) return fail(MPT_EINVAL, "mpt_plan: out is NULL");
  *out = nullptr;
  mpt_path_spec specs[MPT_MAX_PATHS];
  std::memset(specs, 0, sizeof specs);
  const uint32_t mode = ((layout & MPT_PLAN_EAGER) ? 1u : 0u) | ((layout & MPT_PLAN_PAGEABLE) ? MPT_MODE_PAGEABLE : 0u) |
                       ((layout & MPT_PLAN_DUPLEX) ? MPT_MODE_DUPLEX : 0u);
  layout &= ~(MPT_PLAN_EAGER | MPT_PLAN_PAGEABLE | MPT_PLAN_DUPLEX);
  if ((mode & MPT_MODE_PAGEABLE) && dir == MPT_D2D)
    return fail(MPT_EINVAL, "mpt_plan: MPT_PLAN_PAGEABLE needs a host side (H2D or D2H)");
  if ((mode & MPT_MODE_DUPLEX) && (dir == MPT_D2D || (mode & MPT_MODE_PAGEABLE)))
    return fail(MPT_EINVAL, "mpt_plan: MPT_PLAN_DUPLEX needs a host side in page-locked memory");
  if (paths == nullptr) {
    if (align == 0 || (align & (align - 1)) != 0 || align > MPT_MAX_ALIGN)
      return fail(MPT_EINVAL, "mpt_plan: alignment %u is not a power of two <= %u", align, MPT_MAX_ALIGN);
    mpt_status st = tuner_fill(ctx, nbytes, dir, mode, align, specs, &npaths, true);
    if (st != MPT_OK) return st;
  } else {
    if (npaths == 0 || npaths > MPT_MAX_PATHS)
      return fail(MPT_EINVAL, "mpt_plan: need 1..%u paths, got %u", MPT_MAX_PATHS, npaths);
    std::memcpy(specs, paths, npaths * sizeof(mpt_path_spec));
    bool need_tuner = false;
    for (uint32_t p = 0; p < npaths; ++p) need_tuner |= specs[p].chunk_bytes == 0;
    if (need_tuner) {
      if (align == 0 || (align & (align - 1)) != 0 || align > MPT_MAX_ALIGN)
        return fail(MPT_EINVAL, "mpt_plan: alignment %u is not a power of two <= %u", align, MPT_MAX_ALIGN);
      mpt_status st = tuner_fill(ctx, nbytes, dir, mode, align, specs, &npaths, false);
      if (st != MPT_OK) return st;
    }
  }
  mpt_plan_s* plan = new mpt_plan_s;
  mpt_status st = build_chunks(nbytes, dir, specs, npaths, align, layout, plan->chunks, plan->path_bytes);
  if (st != MPT_OK) {
    delete plan;
    return st;
  }
  plan->nbytes = nbytes;
  plan->dir = dir;
  plan->align = align;
  plan->layout = layout;
  plan->npaths = npaths;
  std::memcpy(plan->paths, specs, sizeof specs);
  uint32_t i = 0;
  for (uint32_t p = 0; p <= npaths; ++p) {
    while (i < plan->chunks.size() && plan->chunks[i].path_index < p) ++i;
    plan->first_chunk[p] = i;
  }
  for (uint32_t p = npaths + 1; p <= MPT_MAX_PATHS; ++p) plan->first_chunk[p] = (uint32_t)plan->chunks.size();
  uint64_t h = fnv1a(&nbytes, sizeof nbytes);
  const uint32_t hdr[4] = {dir, align, layout, npaths};
  h = fnv1a(hdr, sizeof hdr, h);
  h = fnv1a(specs, npaths * sizeof(mpt_path_spec), h);
  plan->hash = h;
  *out = plan;
  return MPT_OK;
}

mpt_status mpt_plan_chunks(mpt_plan_t plan, mpt_chunk* out, size_t cap, size_t* n) {
  if (!plan || !n) return fail(MPT_EINVAL, "mpt_plan_chunks: NULL argument");
  if (cap > 0 && !out) return fail(MPT_EINVAL, "mpt_plan_chunks: NULL output with cap %zu", cap);
  const size_t k = plan->chunks.size() < cap ? plan->chunks.size() : cap;
  if (k) std::memcpy(out, plan->chunks.data(), k * sizeof(mpt_chunk));
  *n = plan->chunks.size();
  return MPT_OK;
}

mpt_status mpt_plan_paths(mpt_plan_t plan, mpt_path_spec* out, uint32_t cap, uint32_t* n) {
  if (!plan || !n) return fail(MPT_EINVAL, "mpt_plan_paths: NULL argument");
  if (cap > 0 && !out) return fail(MPT_EINVAL, "mpt_plan_paths: NULL output with cap %u", cap);
  const uint32_t k = plan->npaths < cap ? plan->npaths : cap;
  if (k) std::memcpy(out, plan->paths, k * sizeof(mpt_path_spec));
  *n = plan->npaths;
  return MPT_OK;
}

mpt_status mpt_plan_destroy(mpt_plan_t plan) {
  delete plan;
  return MPT_OK;
}

}  // extern "C"
