// Latency-plus-bandwidth cost model of a multi-path plan and the split search built on it
// (the tuner's starting point; the paper tunes paths and chunks offline by exhaustive
// search over link bandwidths, latencies and message sizes, Sec. 4.4).
//
// Per path p with b_p bytes in k_p = ceil(b_p / C) chunks:
//   T_p  = alpha_p * k_p + ceil(b_p * 1e12 / beta_p)                      (ps)
//   T_HS = alpha * (k + 1) + ceil(b * 1e12 / min(beta1, beta2)) + ceil(min(C, b) * 1e12 / max(beta1, beta2))
// shared resources: T_HBM = ceil(sum h_p b_p 1e12 / B_HBM), T_link,dir = ceil(sum l_p b_p 1e12 / B_link,dir)
// total: T = launch + max(max_p T_p, T_HBM, T_link,h2d, T_link,d2h).
// Integer picoseconds throughout (unsigned __int128 products, ceiling division).
#include <cstring>

#include "internal.h"

namespace mpt {

namespace {

using u128 = unsigned __int128;
constexpr uint64_t kPsPerS = 1000000000000ull;

uint64_t ceil_div128(u128 a, uint64_t b) { return (uint64_t)((a + b - 1) / b); }

const mpt_path_model& model_of(const mpt_model& m, uint32_t kind) {
  switch (kind) {
    case MPT_PATH_CE: return m.ce;
    case MPT_PATH_SM: return m.sm;
    case MPT_PATH_HS: return m.hs;
    default: return m.zc;
  }
}

// HBM crossings and host-link crossings (h2d, d2h) per payload byte.
void crossings(uint32_t dir, uint32_t kind, uint32_t& h, uint32_t& up, uint32_t& down) {
  up = down = 0;
  if (dir == MPT_D2D) {
    h = 2;
    if (kind == MPT_PATH_HS) up = down = 1;
  } else {
    h = kind == MPT_PATH_HS ? 3 : 1;
    (dir == MPT_H2D ? up : down) = 1;
  }
}

uint64_t path_time(const mpt_path_model& pm, uint32_t kind, uint64_t b, uint64_t chunk) {
  if (b == 0) return 0;
  const uint64_t k = (b + chunk - 1) / chunk;
  if (kind == MPT_PATH_HS) {
    const uint64_t slow = pm.beta_Bps < pm.beta2_Bps ? pm.beta_Bps : pm.beta2_Bps;
    const uint64_t fast = pm.beta_Bps < pm.beta2_Bps ? pm.beta2_Bps : pm.beta_Bps;
    const uint64_t first = chunk < b ? chunk : b;
    return pm.alpha_ps * (k + 1) + ceil_div128((u128)b * kPsPerS, slow) + ceil_div128((u128)first * kPsPerS, fast);
  }
  return pm.alpha_ps * k + ceil_div128((u128)b * kPsPerS, pm.beta_Bps);
}

bool model_valid(const mpt_model& m, uint32_t dir, const uint32_t* kinds, uint32_t n) {
  if (m.hbm_Bps == 0 || m.link_h2d_Bps == 0 || m.link_d2h_Bps == 0) return false;
  for (uint32_t p = 0; p < n; ++p) {
    if (!kind_allowed(dir, kinds[p])) return false;
    const mpt_path_model& pm = model_of(m, kinds[p]);
    if (pm.beta_Bps == 0 || (kinds[p] == MPT_PATH_HS && pm.beta2_Bps == 0)) return false;
  }
  return true;
}

}  // namespace

uint64_t model_time(const mpt_model& m, uint32_t dir, const uint32_t* kinds, const uint64_t* bytes, uint32_t n,
                    uint64_t chunk) {
  uint64_t worst = 0;
  u128 hbm = 0, up = 0, down = 0;
  for (uint32_t p = 0; p < n; ++p) {
    const uint64_t t = path_time(model_of(m, kinds[p]), kinds[p], bytes[p], chunk);
    if (t > worst) worst = t;
    uint32_t h, u, d;
    crossings(dir, kinds[p], h, u, d);
    hbm += (u128)h * bytes[p];
    up += (u128)u * bytes[p];
    down += (u128)d * bytes[p];
  }
  uint64_t shared = ceil_div128(hbm * kPsPerS, m.hbm_Bps);
  const uint64_t tu = ceil_div128(up * kPsPerS, m.link_h2d_Bps);
  const uint64_t td = ceil_div128(down * kPsPerS, m.link_d2h_Bps);
  if (tu > shared) shared = tu;
  if (td > shared) shared = td;
  return m.launch_ps + (worst > shared ? worst : shared);
}

// Search every split on a grid (step A for messages up to 4 KiB, so the search is
// exhaustive there; N/64 rounded down to A beyond, i.e. shares in 1/64 steps) and every
// chunk A*2^k <= max(N, A); canonical tie-break: lowest time, fewest non-empty paths,
// lexicographically largest split, largest chunk.
mpt_status model_optimize(const mpt_model& m, uint64_t nbytes, uint32_t dir, const uint32_t* kinds, uint32_t n,
                          uint32_t align, uint64_t* best_bytes, uint64_t* best_chunk, uint64_t* best_ps) {
  if (n == 0 || n > 4) return fail(MPT_EINVAL, "mpt_model_optimize: 1..4 paths");
  if (align == 0 || (align & (align - 1)) || align > MPT_MAX_ALIGN)
    return fail(MPT_EINVAL, "mpt_model_optimize: bad alignment %u", align);
  if (!model_valid(m, dir, kinds, n)) return fail(MPT_EINVAL, "mpt_model_optimize: invalid model or path kinds");
  uint64_t step = align;
  if (nbytes > 4096) {
    step = (nbytes / 64) / align * align;
    if (step < align) step = align;
  }
  bool have = false;
  uint64_t bt = 0, bc = 0, bb[4] = {0, 0, 0, 0};
  uint32_t bn = 0;
  uint64_t cur[4];
  const uint64_t cmax = nbytes > align ? nbytes : align;
  for (uint64_t chunk = align; chunk <= cmax; chunk *= 2) {
    // odometer over b_0..b_{n-2} in multiples of step, last path takes the rest
    uint64_t idx[4] = {0, 0, 0, 0};
    while (true) {
      uint64_t used = 0;
      bool over = false;
      for (uint32_t p = 0; p + 1 < n; ++p) {
        cur[p] = idx[p] * step;
        used += cur[p];
        if (used > nbytes) over = true;
      }
      if (!over) {
        cur[n - 1] = nbytes - used;
        const uint64_t t = model_time(m, dir, kinds, cur, n, chunk);
        uint32_t ne = 0;
        for (uint32_t p = 0; p < n; ++p) ne += cur[p] > 0;
        bool better = !have;
        if (!better) {
          if (t != bt) better = t < bt;
          else if (ne != bn) better = ne < bn;
          else {
            int cmp = 0;
            for (uint32_t p = 0; p < n && cmp == 0; ++p)
              cmp = cur[p] > bb[p] ? 1 : (cur[p] < bb[p] ? -1 : 0);
            if (cmp != 0) better = cmp > 0;
            else better = chunk > bc;
          }
        }
        if (better) {
          have = true;
          bt = t;
          bc = chunk;
          bn = ne;
          std::memcpy(bb, cur, sizeof bb);
        }
      }
      // advance the odometer (skip sums above N)
      int p = (int)n - 2;
      while (p >= 0) {
        idx[p]++;
        uint64_t s = 0;
        for (uint32_t q = 0; q <= (uint32_t)p; ++q) s += idx[q] * step;
        if (s <= nbytes) break;
        idx[p] = 0;
        --p;
      }
      if (p < 0) break;
    }
    if (chunk > cmax / 2) break;
  }
  for (uint32_t p = 0; p < n; ++p) best_bytes[p] = bb[p];
  *best_chunk = bc;
  *best_ps = bt;
  return MPT_OK;
}

}  // namespace mpt

using namespace mpt;

extern "C" {

mpt_status mpt_model_time(const mpt_model* m, uint32_t dir, const uint32_t* kinds, const uint64_t* bytes,
                          uint32_t npaths, uint64_t chunk, uint64_t* out_ps) {
  if (!m || !kinds || !bytes || !out_ps || npaths == 0 || npaths > MPT_MAX_PATHS || chunk == 0)
    return fail(MPT_EINVAL, "mpt_model_time: bad argument");
  if (!model_valid(*m, dir, kinds, npaths)) return fail(MPT_EINVAL, "mpt_model_time: invalid model or path kinds");
  *out_ps = model_time(*m, dir, kinds, bytes, npaths, chunk);
  return MPT_OK;
}

mpt_status mpt_model_optimize(const mpt_model* m, uint64_t nbytes, uint32_t dir, const uint32_t* kinds,
                              uint32_t npaths, uint32_t align, uint64_t* out_bytes, uint64_t* out_chunk,
                              uint64_t* out_ps) {
  if (!m || !kinds || !out_bytes || !out_chunk || !out_ps) return fail(MPT_EINVAL, "mpt_model_optimize: NULL argument");
  return model_optimize(*m, nbytes, dir, kinds, npaths, align, out_bytes, out_chunk, out_ps);
}

}  // extern "C"
