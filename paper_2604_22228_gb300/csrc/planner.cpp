// Chunk planner behind mpt_plan (Sec. 4.3 "2-D Pipelining Engine", Algorithm 1).
//
// Horizontal split: path p < P-1 carries floor_A(floor(N * share_p / 65536)) bytes and
// the last path the remainder.  Vertical split: each path's bytes are cut into chunks of
// chunk_bytes with a short last chunk.  CONTIG lays the paths' regions out back to back
// in path order (Algorithm 1's running sent_data offset); INTERLEAVE deals chunks round by
// round (the round-robin distribution the text after Algorithm 2 describes), deferring the
// one chunk whose length is not a multiple of the alignment to the end of the message.
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace mpt {

namespace {
thread_local std::string g_error;
}

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
}

mpt_status fail(mpt_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return st;
}

const char* last_error_cstr() { return g_error.c_str(); }

bool kind_allowed(uint32_t dir, uint32_t kind) {
  switch (dir) {
    case MPT_D2D:
      return kind == MPT_PATH_CE || kind == MPT_PATH_SM || kind == MPT_PATH_HS;
    case MPT_H2D:
    case MPT_D2H:
      return kind == MPT_PATH_CE || kind == MPT_PATH_ZC || kind == MPT_PATH_HS;
    default:
      return false;
  }
}

uint64_t fnv1a(const void* data, size_t n, uint64_t h) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

mpt_status build_chunks(uint64_t nbytes, uint32_t dir, const mpt_path_spec* paths, uint32_t npaths,
                        uint32_t align, uint32_t layout, std::vector<mpt_chunk>& out,
                        uint64_t* path_bytes) {
  if (dir > MPT_D2H) return fail(MPT_EINVAL, "mpt_plan: unknown direction %u", dir);
  if (layout > MPT_LAYOUT_INTERLEAVE) return fail(MPT_EINVAL, "mpt_plan: unknown layout %u", layout);
  if (align == 0 || (align & (align - 1)) != 0 || align > MPT_MAX_ALIGN)
    return fail(MPT_EINVAL, "mpt_plan: alignment %u is not a power of two <= %u", align, MPT_MAX_ALIGN);
  if (npaths == 0 || npaths > MPT_MAX_PATHS || paths == nullptr)
    return fail(MPT_EINVAL, "mpt_plan: need 1..%u paths, got %u", MPT_MAX_PATHS, npaths);
  uint64_t share_sum = 0;
  for (uint32_t p = 0; p < npaths; ++p) {
    const mpt_path_spec& s = paths[p];
    if (!kind_allowed(dir, s.kind))
      return fail(MPT_EINVAL, "mpt_plan: path %u kind %u cannot carry direction %u", p, s.kind, dir);
    if (s.share == 0) return fail(MPT_EINVAL, "mpt_plan: path %u has a zero share", p);
    if (s.kind == MPT_PATH_HS && (s.flags & MPT_HS_HOST_THREADS) && dir == MPT_D2D)
      return fail(MPT_EINVAL, "mpt_plan: path %u: host-thread staging carries host<->device transfers only", p);
    if (s.chunk_bytes == 0 || s.chunk_bytes % align != 0)
      return fail(MPT_EINVAL, "mpt_plan: path %u chunk %llu is not a positive multiple of %u", p,
                  (unsigned long long)s.chunk_bytes, align);
    share_sum += s.share;
  }
  if (share_sum != MPT_SHARE_ONE)
    return fail(MPT_EINVAL, "mpt_plan: shares sum to %llu, not 65536", (unsigned long long)share_sum);

  // Horizontal split.
  const uint64_t amask = ~(uint64_t)(align - 1);
  uint64_t given = 0;
  for (uint32_t p = 0; p + 1 < npaths; ++p) {
    const unsigned __int128 scaled = (unsigned __int128)nbytes * paths[p].share;
    path_bytes[p] = (uint64_t)(scaled >> 16) & amask;
    given += path_bytes[p];
  }
  path_bytes[npaths - 1] = nbytes - given;

  // Vertical split: chunk counts and where each path's chunks start in the output.
  uint64_t count[MPT_MAX_PATHS], first[MPT_MAX_PATHS + 1];
  first[0] = 0;
  uint64_t most = 0;
  for (uint32_t p = 0; p < npaths; ++p) {
    count[p] = (path_bytes[p] + paths[p].chunk_bytes - 1) / paths[p].chunk_bytes;
    first[p + 1] = first[p] + count[p];
    if (count[p] > most) most = count[p];
  }
  if (first[npaths] > MPT_MAX_CHUNKS)
    return fail(MPT_EINVAL, "mpt_plan: %llu chunks exceed the limit of %u",
                (unsigned long long)first[npaths], MPT_MAX_CHUNKS);
  out.assign(first[npaths], mpt_chunk{});

  auto chunk_len = [&](uint32_t p, uint64_t j) {
    const uint64_t c = paths[p].chunk_bytes;
    return j + 1 < count[p] ? c : path_bytes[p] - j * c;
  };

  if (layout == MPT_LAYOUT_CONTIG) {
    uint64_t region = 0;
    for (uint32_t p = 0; p < npaths; ++p) {
      for (uint64_t j = 0; j < count[p]; ++j)
        out[first[p] + j] = mpt_chunk{region + j * paths[p].chunk_bytes, chunk_len(p, j), p, (uint32_t)j};
      region += path_bytes[p];
    }
  } else {
    const uint32_t last = npaths - 1;
    const bool ragged = path_bytes[last] % align != 0;
    uint64_t cursor = 0;
    for (uint64_t round = 0; round < most; ++round) {
      for (uint32_t p = 0; p < npaths; ++p) {
        if (round >= count[p]) continue;
        if (p == last && ragged && round + 1 == count[p]) continue;  // placed at the end
        const uint64_t len = chunk_len(p, round);
        out[first[p] + round] = mpt_chunk{cursor, len, p, (uint32_t)round};
        cursor += len;
      }
    }
    if (ragged) {
      const uint64_t j = count[last] - 1;
      out[first[last] + j] = mpt_chunk{cursor, chunk_len(last, j), last, (uint32_t)j};
      cursor += chunk_len(last, j);
    }
    if (cursor != nbytes) return fail(MPT_EINVAL, "mpt_plan: internal error, plan covers %llu of %llu bytes",
                                      (unsigned long long)cursor, (unsigned long long)nbytes);
  }
  return MPT_OK;
}

}  // namespace mpt
