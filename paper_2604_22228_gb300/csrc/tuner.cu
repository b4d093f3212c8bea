// Autotuner: chooses the path set, shares, chunk size and CTA count for a message, cached
// per (direction, execution mode, log2 size bucket).  Sec. 4.4: paths and chunks can be
// set through environment variables, otherwise tuned values found by an offline search
// are the defaults, kept separately for graph and non-graph execution.
//
//  * environment (highest priority): MPT_PATHS=ce,sm,hs,zc (path kinds in order),
//    MPT_SHARES=w0,w1,... (parts of 65536; default equal), MPT_CHUNK_BYTES=C or
//    MPT_CHUNKS=k (chunks per path), MPT_CTAS=n, MPT_SM_VARIANT=vec|bulk;
//  * a measured entry for the bucket (mpt_tune, or loaded from a tune file);
//  * otherwise the cost model's best split (mpt_model_optimize) with parameters measured
//    on GB300 (default_model).
#include <algorithm>
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "ctx.h"

#define CUDA_TRY(expr)                                                                           \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return mpt::fail(MPT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

namespace mpt {

// Implemented in runtime.cu: build a private (uncached) graph / run eagerly.
mpt_status build_private_graph(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, mpt_graph_s* g);
void free_private_graph(mpt_graph_s* g);
mpt_status run_eager(mpt_ctx_t c, const mpt_plan_s* plan, void* dst, const void* src, cudaStream_t s);

uint32_t size_bucket(uint64_t n) { return n == 0 ? 0u : 63u - (uint32_t)__builtin_clzll(n); }

// Cost-model parameters from measurements on a GB300 (152 SMs, 3 copy engines): SM copy
// and copy-engine device copies near 3.3 TB/s of payload (6.6-6.8 TB/s of HBM traffic);
// host link about 211 GB/s host-to-device and 193 GB/s device-to-host for copy engines
// and the zero-copy kernel alike; a few microseconds of issue cost per memcpy.
mpt_model default_model(uint32_t dir, uint32_t mode) {
  mpt_model m{};
  const uint64_t us = 1000000;  // ps per microsecond
  m.launch_ps = mode == 0 ? 3 * us : 2 * us;
  m.hbm_Bps = 6757900000000ull;
  m.link_h2d_Bps = 211000000000ull;
  m.link_d2h_Bps = 193000000000ull;
  const uint64_t link = dir == MPT_D2H ? m.link_d2h_Bps : m.link_h2d_Bps;
  if (dir == MPT_D2D) {
    m.ce = mpt_path_model{(mode == 0 ? 2 : 4) * us, 3380000000000ull, 0};
    m.sm = mpt_path_model{mode == 0 ? us / 2 : us, 3400000000000ull, 0};
    m.hs = mpt_path_model{(mode == 0 ? 3 : 5) * us, m.link_d2h_Bps, m.link_h2d_Bps};
    m.zc = mpt_path_model{us, link, 0};
  } else {
    m.ce = mpt_path_model{(mode == 0 ? 2 : 4) * us, link, 0};
    m.zc = mpt_path_model{mode == 0 ? us / 2 : us, link, 0};
    m.hs = mpt_path_model{(mode == 0 ? 3 : 5) * us, link, 3400000000000ull};
    m.sm = mpt_path_model{us, 3400000000000ull, 0};
  }
  return m;
}

namespace {

uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

uint32_t parse_kind(const std::string& s) {
  if (s == "ce") return MPT_PATH_CE;
  if (s == "sm") return MPT_PATH_SM;
  if (s == "hs") return MPT_PATH_HS;
  if (s == "zc") return MPT_PATH_ZC;
  return 0;
}

std::vector<std::string> split_list(const char* v) {
  std::vector<std::string> out;
  std::string cur;
  for (const char* p = v; *p; ++p) {
    if (*p == ',') {
      out.push_back(cur);
      cur.clear();
    } else if (*p != ' ') {
      cur += (char)std::tolower((unsigned char)*p);
    }
  }
  out.push_back(cur);
  return out;
}

bool env_u64(const char* name, uint64_t& out) {
  const char* v = std::getenv(name);
  if (!v || !*v) return false;
  char* end = nullptr;
  errno = 0;
  unsigned long long x = std::strtoull(v, &end, 0);
  if (errno || !end || *end) return false;
  out = x;
  return true;
}

// Shares for byte counts: w_p = floor(65536 * b_p / N) for p < P-1, remainder last;
// paths that would get no share are dropped.
uint32_t specs_from_bytes(uint64_t n, const uint32_t* kinds, const uint64_t* bytes, uint32_t np, uint64_t chunk,
                          mpt_path_spec* out) {
  uint32_t k = 0;
  uint64_t given = 0;
  uint64_t nonempty = 0;
  for (uint32_t p = 0; p < np; ++p) nonempty += bytes[p] > 0;
  if (n == 0 || nonempty <= 1) {
    uint32_t p = 0;
    while (p + 1 < np && bytes[p] == 0) ++p;
    out[0] = mpt_path_spec{kinds[p], MPT_SHARE_ONE, chunk, 0, 0};
    return 1;
  }
  for (uint32_t p = 0; p < np; ++p) {
    if (bytes[p] == 0) continue;
    uint64_t w = (uint64_t)(((unsigned __int128)bytes[p] * MPT_SHARE_ONE) / n);
    if (w == 0) w = 1;
    out[k++] = mpt_path_spec{kinds[p], (uint32_t)w, chunk, 0, 0};
    given += w;
  }
  // the last listed path absorbs rounding so shares sum to 65536
  int64_t fix = (int64_t)MPT_SHARE_ONE - (int64_t)given;
  out[k - 1].share = (uint32_t)((int64_t)out[k - 1].share + fix);
  if ((int32_t)out[k - 1].share <= 0) {
    out[k - 1].share = 1;
    uint64_t s = 0;
    for (uint32_t p = 0; p + 1 < k; ++p) s += out[p].share;
    out[0].share -= (uint32_t)(s + 1 - MPT_SHARE_ONE);
  }
  return k;
}

TuneEntry model_choice(uint64_t n, uint32_t dir, uint32_t mode, uint32_t align) {
  const mpt_model m = default_model(dir, mode);
  static const uint32_t d2d_sets[3][2] = {{MPT_PATH_SM, 0}, {MPT_PATH_CE, 0}, {MPT_PATH_CE, MPT_PATH_SM}};
  static const uint32_t host_sets[3][2] = {{MPT_PATH_CE, 0}, {MPT_PATH_ZC, 0}, {MPT_PATH_CE, MPT_PATH_ZC}};
  const uint32_t(*sets)[2] = dir == MPT_D2D ? d2d_sets : host_sets;
  TuneEntry best;
  uint64_t best_t = ~0ull;
  for (int s = 0; s < 3; ++s) {
    const uint32_t np = sets[s][1] ? 2 : 1;
    uint64_t bytes[2], chunk, t;
    if (model_optimize(m, n, dir, sets[s], np, align, bytes, &chunk, &t) != MPT_OK) continue;
    if (t < best_t) {
      best_t = t;
      best.npaths = specs_from_bytes(n, sets[s], bytes, np, chunk, best.paths);
      best.us = (double)t / 1e6;
    }
  }
  return best;
}

// Untuned choice for pageable host memory: the zero-copy kernel alone where the device
// reaches pageable memory (it runs at the host link's speed on a coherent host), else
// host-thread staging with the largest stage chunk.
TuneEntry pageable_default(mpt_ctx_t c, uint64_t n, uint32_t align) {
  TuneEntry e;
  e.npaths = 1;
  const uint64_t whole = std::max<uint64_t>(align, round_up(std::max<uint64_t>(n, 1), align));
  if (c->pageable) {
    e.paths[0] = mpt_path_spec{MPT_PATH_ZC, MPT_SHARE_ONE, whole, 0, 0};
  } else {
    e.paths[0] = mpt_path_spec{MPT_PATH_HS, MPT_SHARE_ONE, std::min<uint64_t>(whole, c->stage_max / align * align), 0,
                               MPT_HS_HOST_THREADS};
  }
  return e;
}

// MPT_PATHS and friends; false when MPT_PATHS is unset.
bool env_choice(uint64_t n, uint32_t dir, uint32_t align, TuneEntry& e, mpt_status& st) {
  const char* pv = std::getenv("MPT_PATHS");
  st = MPT_OK;
  if (!pv || !*pv) return false;
  std::vector<std::string> names = split_list(pv);
  if (names.empty() || names.size() > 4) {
    st = fail(MPT_EINVAL, "MPT_PATHS: 1..4 paths");
    return true;
  }
  e = TuneEntry{};
  e.npaths = (uint32_t)names.size();
  std::vector<uint32_t> shares(e.npaths, 0);
  const char* sv = std::getenv("MPT_SHARES");
  if (sv && *sv) {
    std::vector<std::string> ws = split_list(sv);
    if (ws.size() != names.size()) {
      st = fail(MPT_EINVAL, "MPT_SHARES: %zu values for %zu paths", ws.size(), names.size());
      return true;
    }
    for (size_t i = 0; i < ws.size(); ++i) shares[i] = (uint32_t)std::strtoul(ws[i].c_str(), nullptr, 0);
  } else {
    for (uint32_t p = 0; p < e.npaths; ++p) shares[p] = MPT_SHARE_ONE / e.npaths;
    shares[e.npaths - 1] += MPT_SHARE_ONE % e.npaths;
  }
  uint64_t chunk = 0, nchunks = 0, ctas = 0;
  env_u64("MPT_CHUNK_BYTES", chunk);
  env_u64("MPT_CHUNKS", nchunks);
  env_u64("MPT_CTAS", ctas);
  const char* var = std::getenv("MPT_SM_VARIANT");
  const uint32_t flags = (var && std::strcmp(var, "bulk") == 0) ? MPT_SM_BULK : MPT_SM_VEC128;
  for (uint32_t p = 0; p < e.npaths; ++p) {
    const uint32_t kind = parse_kind(names[p]);
    if (!kind) {
      st = fail(MPT_EINVAL, "MPT_PATHS: unknown path '%s' (ce, sm, hs, zc)", names[p].c_str());
      return true;
    }
    uint64_t c = chunk;
    if (!c) {
      const uint64_t bp = (uint64_t)(((unsigned __int128)n * shares[p]) >> 16);
      c = nchunks ? (bp + nchunks - 1) / nchunks : (4ull << 20);
    }
    c = std::max<uint64_t>(align, round_up(c, align));
    e.paths[p] = mpt_path_spec{kind, shares[p], c, (uint32_t)ctas, kind == MPT_PATH_SM ? flags : 0u};
  }
  return true;
}

mpt_status ensure_dev(void*& p, uint64_t& have, uint64_t need) {
  if (have >= need) return MPT_OK;
  if (p) cudaFree(p);
  p = nullptr;
  have = 0;
  CUDA_TRY(cudaMalloc(&p, need));
  have = need;
  return MPT_OK;
}

}  // namespace

mpt_status tuner_fill(mpt_ctx_t ctx, uint64_t nbytes, uint32_t dir, uint32_t mode, uint32_t align,
                      mpt_path_spec* specs, uint32_t* npaths, bool whole_set) {
  if (dir > MPT_D2H) return fail(MPT_EINVAL, "mpt_plan: unknown direction %u", dir);
  TuneEntry e;
  mpt_status st;
  bool from_env = env_choice(nbytes, dir, align, e, st);
  if (st != MPT_OK) return st;
  if (!from_env) {
    if (!ctx) return fail(MPT_EINVAL, "mpt_plan: the tuner needs a context (or MPT_PATHS)");
    auto it = ctx->tuned.find(tune_key(dir, mode, size_bucket(nbytes)));
    if (it != ctx->tuned.end()) {
      e = it->second;
    } else if (mode & MPT_MODE_PAGEABLE) {
      e = pageable_default(ctx, nbytes, align);
    } else if (mode & MPT_MODE_DUPLEX) {  // one copy-engine chunk: the best measured pair
      e = TuneEntry{};
      e.npaths = 1;
      e.paths[0] = mpt_path_spec{MPT_PATH_CE, MPT_SHARE_ONE, std::max<uint64_t>(align, round_up(nbytes, align)), 0, 0};
    } else {
      e = model_choice(nbytes, dir, mode, align);
    }
  }
  for (uint32_t p = 0; p < e.npaths; ++p) e.paths[p].chunk_bytes = std::max<uint64_t>(align, round_up(e.paths[p].chunk_bytes, align));
  if (whole_set) {
    std::memcpy(specs, e.paths, e.npaths * sizeof(mpt_path_spec));
    *npaths = e.npaths;
    return MPT_OK;
  }
  for (uint32_t p = 0; p < *npaths; ++p) {
    if (specs[p].chunk_bytes) continue;
    uint64_t c = 0;
    for (uint32_t q = 0; q < e.npaths && !c; ++q)
      if (e.paths[q].kind == specs[p].kind) c = e.paths[q].chunk_bytes;
    if (!c) c = e.npaths ? e.paths[0].chunk_bytes : (4ull << 20);
    specs[p].chunk_bytes = std::max<uint64_t>(align, round_up(c, align));
  }
  return MPT_OK;
}

namespace {

constexpr uint64_t kChainMaxBytes = 64ull << 20;  // messages timed as launch chains
constexpr uint32_t kChainLaunches = 8;             // launches per chain, one buffer region each

struct Candidate {
  uint32_t n;
  mpt_path_spec p[4];
};

std::vector<Candidate> candidates(mpt_ctx_t c, uint32_t dir, uint64_t n, uint32_t mode) {
  std::vector<Candidate> out;
  const uint32_t sms = (uint32_t)c->sms;
  // chunk sizes of 64 KiB and more are rounded up to 64 KiB multiples: copy engines move
  // chunks whose boundaries are not page-aligned at about half speed (GB300, 3 x 21.33 MiB:
  // 51 us against 27 us for 3 x 21.375 MiB)
  auto chunk_for = [](uint64_t bytes, uint64_t parts) {
    const uint64_t c = (bytes + parts - 1) / std::max<uint64_t>(parts, 1);
    return std::max<uint64_t>(16, c >= (64u << 10) ? round_up(c, 64u << 10) : round_up(c, 16));
  };
  auto one = [&](uint32_t kind, uint64_t chunk, uint32_t ctas, uint32_t flags) {
    Candidate k{};
    k.n = 1;
    k.p[0] = mpt_path_spec{kind, MPT_SHARE_ONE, chunk, ctas, flags};
    out.push_back(k);
  };
  auto two = [&](uint32_t k0, uint32_t w0, uint64_t c0, uint32_t k1, uint64_t c1, uint32_t ctas1, uint32_t f1) {
    Candidate k{};
    k.n = 2;
    k.p[0] = mpt_path_spec{k0, w0, c0, 0, 0};
    k.p[1] = mpt_path_spec{k1, MPT_SHARE_ONE - w0, c1, ctas1, f1};
    out.push_back(k);
  };
  const uint64_t whole = chunk_for(n, 1);
  if (mode & MPT_MODE_PAGEABLE) {
    // paths that accept pageable host memory: zero-copy (where the device reaches it) and
    // host-thread staging, alone and split
    const uint64_t smax = c->stage_max / 16 * 16;
    if (c->pageable)
      for (uint32_t ctas : {sms / 2, sms, 2 * sms}) one(MPT_PATH_ZC, whole, ctas, 0);
    for (uint64_t cb : {2ull << 20, 4ull << 20, 8ull << 20}) {
      const uint64_t ch = std::min<uint64_t>(std::min(cb, smax), whole);
      one(MPT_PATH_HS, ch, 0, MPT_HS_HOST_THREADS);
      if (ch >= whole) break;
    }
    if (c->pageable && n >= (4u << 20)) {
      for (uint32_t w : {32768u, 49152u, 57344u}) {
        Candidate k{};
        k.n = 2;
        k.p[0] = mpt_path_spec{MPT_PATH_ZC, w, chunk_for((n * w) >> 16, 1), sms, 0};
        k.p[1] = mpt_path_spec{MPT_PATH_HS, MPT_SHARE_ONE - w, std::min<uint64_t>(smax, whole), 0,
                               MPT_HS_HOST_THREADS};
        out.push_back(k);
      }
    }
    return out;
  }
  if (dir == MPT_D2D) {
    for (uint32_t ctas : {sms, 4 * sms, 16 * sms, 64 * sms}) one(MPT_PATH_SM, whole, ctas, MPT_SM_VEC128);
    if (n <= (32ull << 20) && n > (64u << 10))
      for (uint32_t ctas : {4 * sms, 16 * sms}) one(MPT_PATH_SM, whole, ctas, MPT_SM_TILE8K);
    if (n >= (1u << 20))  // the bulk kernel, many waves of its resident CTAs
      for (uint32_t ctas : {16 * sms, 32 * sms}) one(MPT_PATH_SM, whole, ctas, MPT_SM_BULK);
    for (uint64_t parts : {1, 2, 3, 4, 8}) {
      if (parts > 1 && n < parts * (64u << 10)) continue;
      one(MPT_PATH_CE, chunk_for(n, parts), 0, 0);
    }
    if (n >= (256u << 10)) {
      for (uint32_t w : {4096u, 8192u, 16384u, 24576u, 32768u, 40960u, 49152u})
        for (uint64_t parts : {1, 2, 4}) {
          const uint64_t bce = (n * w) >> 16;
          two(MPT_PATH_CE, w, chunk_for(bce, parts), MPT_PATH_SM, chunk_for(n - bce, 1), 16 * sms, MPT_SM_VEC128);
        }
    }
  } else {
    for (uint64_t parts : {1, 2, 4, 8}) {
      if (parts > 1 && n < parts * (64u << 10)) continue;
      one(MPT_PATH_CE, chunk_for(n, parts), 0, 0);
    }
    for (uint32_t ctas : {sms / 2, sms, 2 * sms}) one(MPT_PATH_ZC, whole, ctas, 0);
    if (n >= (256u << 10)) {
      for (uint32_t w : {16384u, 32768u, 49152u, 57344u})
        for (uint64_t parts : {1, 4}) {
          const uint64_t bce = (n * w) >> 16;
          two(MPT_PATH_CE, w, chunk_for(bce, parts), MPT_PATH_ZC, chunk_for(n - bce, 1), sms, 0);
        }
    }
    if (n >= (1u << 20))
      for (uint64_t cb : {1ull << 20, 4ull << 20, 8ull << 20})
        if (cb <= c->stage_max && cb <= n) one(MPT_PATH_HS, cb, 0, 0);
  }
  return out;
}

}  // namespace

}  // namespace mpt

using namespace mpt;

extern "C" {

mpt_status mpt_tune(mpt_ctx_t c, uint32_t dir, uint64_t nbytes, uint32_t mode, uint32_t reps, mpt_path_spec* out,
                    uint32_t* out_n, double* out_us) {
  if (!c) return fail(MPT_EINVAL, "mpt_tune: NULL context");
  const bool pageable = (mode & MPT_MODE_PAGEABLE) != 0;
  const bool duplex = (mode & MPT_MODE_DUPLEX) != 0;
  const bool graph_mode = (mode & 1u) == 0;
  if (dir > MPT_D2H || (mode & ~(MPT_MODE_PAGEABLE | MPT_MODE_DUPLEX)) > 1 || (pageable && dir == MPT_D2D) ||
      (duplex && (dir == MPT_D2D || pageable)))
    return fail(MPT_EINVAL, "mpt_tune: bad direction or mode");
  if (nbytes == 0) return fail(MPT_EINVAL, "mpt_tune: empty message");
  if (reps == 0) reps = nbytes >= (256ull << 20) ? 3 : (nbytes >= (16ull << 20) ? 5 : 11);
  CUDA_TRY(cudaSetDevice(c->device));
  // A message of at most 64 MiB is timed as a chain of back-to-back launches, each on its own
  // buffer region (no launch finds the previous one's data in L2): in a stream of messages
  // the fixed cost of a launch overlaps the copy before it (programmatic dependent launch of
  // the copy kernels; copy engines queue their work), which a single launch after the flush
  // cannot show, and a graph launch does not overlap that way.
  const uint32_t chain = nbytes <= kChainMaxBytes ? kChainLaunches : 1u;
  const uint64_t stride = (nbytes + 4095) / 4096 * 4096;
  const uint64_t span = chain == 1 ? nbytes : chain * stride;
  // buffers: device a/b, page-locked host h, and a 256 MiB L2 flush buffer
  mpt_status st = ensure_dev(c->tune_a, c->tune_dev_bytes, span);
  if (st != MPT_OK) return st;
  if (c->tune_b) cudaFree(c->tune_b);
  c->tune_b = nullptr;
  CUDA_TRY(cudaMalloc(&c->tune_b, c->tune_dev_bytes));
  if (pageable && c->tune_pg_bytes < span) {
    std::free(c->tune_pg);
    c->tune_pg = std::malloc(span);
    if (!c->tune_pg) {
      c->tune_pg_bytes = 0;
      return fail(MPT_ENOMEM, "mpt_tune: pageable host buffer of %llu bytes", (unsigned long long)span);
    }
    std::memset(c->tune_pg, 0x5a, span);  // touch every page before timing
    c->tune_pg_bytes = span;
  }
  if (!pageable && dir != MPT_D2D && c->tune_host_bytes < span) {
    if (c->tune_h) cudaFreeHost(c->tune_h);
    c->tune_h = nullptr;
    c->tune_host_bytes = 0;
    CUDA_TRY(cudaHostAlloc(&c->tune_h, span, cudaHostAllocMapped | cudaHostAllocPortable));
    c->tune_host_bytes = span;
  }
  if (duplex && c->tune_h2_bytes < span) {  // the opposite direction's host side
    if (c->tune_h2) cudaFreeHost(c->tune_h2);
    c->tune_h2 = nullptr;
    c->tune_h2_bytes = 0;
    CUDA_TRY(cudaHostAlloc(&c->tune_h2, span, cudaHostAllocPortable));
    c->tune_h2_bytes = span;
  }
  st = ensure_dev(c->flush, c->flush_bytes, 256ull << 20);
  if (st != MPT_OK) return st;
  void* host = pageable ? c->tune_pg : c->tune_h;
  void* src = dir == MPT_H2D ? host : c->tune_a;
  void* dst = dir == MPT_D2H ? host : c->tune_b;
  // duplex: the mirrored plan runs device -> second host buffer beside a host-to-device
  // candidate, second host buffer -> the device buffer a device-to-host candidate leaves unused
  void* opp_src = dir == MPT_H2D ? c->tune_a : c->tune_h2;
  void* opp_dst = dir == MPT_H2D ? c->tune_h2 : c->tune_b;
  cudaStream_t s = c->lane[MPT_MAX_PATHS - 1].s[0];
  cudaStream_t s_opp = c->lane[MPT_MAX_PATHS - 1].s[1];
  cudaEvent_t e0, e1, e_opp;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  CUDA_TRY(cudaEventCreateWithFlags(&e_opp, cudaEventDisableTiming));
  TuneEntry best;
  double best_us = 1e30;
  auto region = [&](void* base, uint32_t k) -> void* { return static_cast<uint8_t*>(base) + (uint64_t)k * stride; };
  const char* vv = std::getenv("MPT_TUNE_VERBOSE");
  const bool verbose = vv && *vv && *vv != '0';
  // One candidate ready to run: its plan (and the mirrored plan for duplex timing), and in
  // graph mode one private graph per buffer region of the chain.
  struct Run {
    Candidate k{};
    mpt_plan_t plan = nullptr, mirror = nullptr;
    std::vector<mpt_graph_s> g, gm;
    std::vector<float> ts;  // per-launch ms of each timed run
  };
  auto close_run = [&](Run& R) {
    for (mpt_graph_s& gk : R.g) free_private_graph(&gk);
    for (mpt_graph_s& gk : R.gm) free_private_graph(&gk);
    R.g.clear();
    R.gm.clear();
    if (R.plan) mpt_plan_destroy(R.plan);
    if (R.mirror) mpt_plan_destroy(R.mirror);
    R.plan = R.mirror = nullptr;
  };
  auto open_run = [&](const Candidate& k, Run& R) -> bool {
    R.k = k;
    if (mpt_plan(nullptr, nbytes, dir, k.p, k.n, 16, MPT_LAYOUT_CONTIG, &R.plan) != MPT_OK) return false;
    // duplex: the same path set in the opposite direction runs at the same time (the paper's
    // bidirectional test moves equal messages both ways), and the time is until both finish
    if (duplex && mpt_plan(nullptr, nbytes, dir == MPT_H2D ? MPT_D2H : MPT_H2D, k.p, k.n, 16, MPT_LAYOUT_CONTIG,
                           &R.mirror) != MPT_OK) {
      close_run(R);
      return false;
    }
    R.g.resize(graph_mode ? chain : 0);
    R.gm.resize(graph_mode && duplex ? chain : 0);
    bool ok = true;
    for (uint32_t k2 = 0; ok && k2 < R.g.size(); ++k2)
      ok = build_private_graph(c, R.plan, region(dst, k2), region(src, k2), &R.g[k2]) == MPT_OK;
    for (uint32_t k2 = 0; ok && k2 < R.gm.size(); ++k2)
      ok = build_private_graph(c, R.mirror, region(opp_dst, k2), region(opp_src, k2), &R.gm[k2]) == MPT_OK;
    if (!ok) close_run(R);
    return ok;
  };
  // One timed run: write 256 MiB (twice the L2) first, on the timing stream, so that each run
  // starts with a cold L2 full of dirty lines, as after the kernel that produced the data;
  // then the chain of launches.  Returns false when a launch or the synchronisation failed.
  auto run_once = [&](Run& R, uint32_t r, bool keep) -> bool {
    bool ok = true;
    cudaMemsetAsync(c->flush, r & 0xff, c->flush_bytes, s);
    cudaEventRecord(e0, s);
    if (duplex) cudaStreamWaitEvent(s_opp, e0, 0);
    for (uint32_t k2 = 0; ok && k2 < chain; ++k2) {
      if (graph_mode) ok = R.g[k2].exec == nullptr || cudaGraphLaunch(R.g[k2].exec, s) == cudaSuccess;
      else ok = run_eager(c, R.plan, region(dst, k2), region(src, k2), s) == MPT_OK;
      if (ok && duplex) {
        if (graph_mode) ok = R.gm[k2].exec == nullptr || cudaGraphLaunch(R.gm[k2].exec, s_opp) == cudaSuccess;
        else ok = run_eager(c, R.mirror, region(opp_dst, k2), region(opp_src, k2), s_opp) == MPT_OK;
      }
    }
    if (duplex) {
      cudaEventRecord(e_opp, s_opp);
      cudaStreamWaitEvent(s, e_opp, 0);
    }
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) ok = false;
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ok && keep) R.ts.push_back(ms / (float)chain);
    return ok;
  };
  auto median_us = [](std::vector<float> v) {
    std::sort(v.begin(), v.end());
    return 1e3 * v[v.size() / 2];
  };
  auto log_run = [&](const char* tag, const Run& R, double us) {
    if (!verbose) return;
    std::fprintf(stderr, "mpt_tune%s dir=%u mode=%u n=%llu us=%.2f min=%.2f max=%.2f paths=", tag, dir, mode,
                 (unsigned long long)nbytes, us, 1e3 * *std::min_element(R.ts.begin(), R.ts.end()),
                 1e3 * *std::max_element(R.ts.begin(), R.ts.end()));
    for (uint32_t p = 0; p < R.k.n; ++p)
      std::fprintf(stderr, "[%u %u %llu %u %u]", R.k.p[p].kind, R.k.p[p].share,
                   (unsigned long long)R.k.p[p].chunk_bytes, R.k.p[p].ctas, R.k.p[p].flags);
    std::fprintf(stderr, "\n");
  };
  auto keep_if_best = [&](const Candidate& k, double us) {
    if (us < best_us) {
      best_us = us;
      best = TuneEntry{};
      best.npaths = k.n;
      std::memcpy(best.paths, k.p, sizeof k.p);
      best.us = us;
    }
  };
  struct Timed {
    Candidate k;
    double us;
  };
  std::vector<Timed> timed;  // every candidate that ran, with its median
  auto measure = [&](const Candidate& k) {
    Run R;
    if (!open_run(k, R)) {
      cudaGetLastError();
      return;
    }
    bool ok = true;
    for (uint32_t r = 0; ok && r < reps + 1; ++r) ok = run_once(R, r, r > 0);  // the first run warms up
    close_run(R);
    if (!ok || R.ts.empty()) {
      cudaGetLastError();
      return;
    }
    const double us = median_us(R.ts);
    log_run("", R, us);
    timed.push_back(Timed{k, us});
    keep_if_best(k, us);
  };
  for (const Candidate& k : candidates(c, dir, nbytes, mode)) measure(k);
  // A two-path winner is refined in 1/64 steps of the message around its share (the coarse
  // list steps by 1/16 .. 1/8); chunk sizes, CTAs and variants stay as they won.
  if (best.npaths == 2) {
    const TuneEntry coarse = best;
    for (int step : {-2, -1, 1, 2}) {
      const int64_t w = (int64_t)coarse.paths[0].share + step * (int64_t)(MPT_SHARE_ONE / 64);
      if (w <= 0 || w >= (int64_t)MPT_SHARE_ONE) continue;
      Candidate k{};
      k.n = 2;
      k.p[0] = coarse.paths[0];
      k.p[1] = coarse.paths[1];
      k.p[0].share = (uint32_t)w;
      k.p[1].share = MPT_SHARE_ONE - (uint32_t)w;
      measure(k);
    }
  }
  // Confirmation.  The candidates above ran one after another, each over a few runs, and the
  // lowest of some forty medians is biased low (the winner's curse); the host link and HBM
  // also drift between the first candidate and the last.  The three leaders and the fastest
  // single-path candidate of each path kind are therefore timed again in interleaved rounds
  // (one run of each per round, after one warm-up round), and the lowest median of those
  // rounds is the choice: a split is kept only where it beats the best single path in the
  // same rounds.
  if (timed.size() > 1) {
    std::vector<size_t> order(timed.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return timed[a].us < timed[b].us; });
    std::vector<size_t> pick;
    for (size_t i = 0; i < order.size() && pick.size() < 3; ++i) pick.push_back(order[i]);
    for (uint32_t kind : {MPT_PATH_CE, MPT_PATH_SM, MPT_PATH_HS, MPT_PATH_ZC})
      for (size_t i : order)
        if (timed[i].k.n == 1 && timed[i].k.p[0].kind == kind) {
          if (std::find(pick.begin(), pick.end(), i) == pick.end()) pick.push_back(i);
          break;
        }
    std::vector<Run> runs(pick.size());
    std::vector<bool> live(pick.size(), false);
    for (size_t j = 0; j < pick.size(); ++j) live[j] = open_run(timed[pick[j]].k, runs[j]);
    const uint32_t rounds = std::max<uint32_t>(reps, 5);
    for (uint32_t r = 0; r < rounds + 1; ++r)
      for (size_t j = 0; j < runs.size(); ++j)
        if (live[j]) live[j] = run_once(runs[j], r, r > 0);
    best_us = 1e30;
    best = TuneEntry{};
    for (size_t j = 0; j < runs.size(); ++j) {
      if (live[j] && !runs[j].ts.empty()) {
        const double us = median_us(runs[j].ts);
        log_run(" confirm", runs[j], us);
        keep_if_best(runs[j].k, us);
      }
      close_run(runs[j]);
    }
    cudaGetLastError();
    if (best.npaths == 0)  // nothing ran again: keep the first pass's choice
      keep_if_best(timed[order[0]].k, timed[order[0]].us);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e_opp);
  if (best.npaths == 0) return fail(MPT_ECUDA, "mpt_tune: no candidate ran");
  mpt_status dev = mpt_ctx_status(c, nullptr);
  if (dev != MPT_OK) return dev;
  c->tuned[tune_key(dir, mode, size_bucket(nbytes))] = best;
  if (out) std::memcpy(out, best.paths, best.npaths * sizeof(mpt_path_spec));
  if (out_n) *out_n = best.npaths;
  if (out_us) *out_us = best.us;
  return MPT_OK;
}

mpt_status mpt_tune_save(mpt_ctx_t c, const char* path) {
  if (!c || !path) return fail(MPT_EINVAL, "mpt_tune_save: NULL argument");
  FILE* f = std::fopen(path, "w");
  if (!f) return fail(MPT_EINVAL, "mpt_tune_save: cannot open %s", path);
  for (const auto& kv : c->tuned) {
    const TuneEntry& e = kv.second;
    std::fprintf(f, "{\"dir\": %u, \"mode\": %u, \"bucket\": %u, \"layout\": %u, \"us\": %.3f, \"paths\": [",
                 kv.first >> 16, (kv.first >> 8) & 0xffu, kv.first & 0xffu, e.layout, e.us);
    for (uint32_t p = 0; p < e.npaths; ++p)
      std::fprintf(f, "%s[%u, %u, %llu, %u, %u]", p ? ", " : "", e.paths[p].kind, e.paths[p].share,
                   (unsigned long long)e.paths[p].chunk_bytes, e.paths[p].ctas, e.paths[p].flags);
    std::fprintf(f, "]}\n");
  }
  std::fclose(f);
  return MPT_OK;
}

// Reads the JSON-lines file mpt_tune_save writes (numbers in its fixed key order).
mpt_status mpt_tune_load(mpt_ctx_t c, const char* path) {
  if (!c || !path) return fail(MPT_EINVAL, "mpt_tune_load: NULL argument");
  FILE* f = std::fopen(path, "r");
  if (!f) return fail(MPT_EINVAL, "mpt_tune_load: cannot open %s", path);
  char line[1024];
  uint32_t lineno = 0;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (line[0] == '#') continue;  // comment lines (e.g. the device the table was tuned on)
    double v[5 + 5 * 4];
    int n = 0;
    for (char* p = line; *p && n < (int)(sizeof v / sizeof v[0]);) {
      if ((*p >= '0' && *p <= '9') || (*p == '-' && p[1] >= '0' && p[1] <= '9')) {
        char* end;
        v[n++] = std::strtod(p, &end);
        p = end;
      } else {
        ++p;
      }
    }
    if (n == 0) continue;
    const uint32_t lmode = (uint32_t)v[1];
    if (n < 10 || (n - 5) % 5 != 0 || v[0] > 2 || (lmode & ~(MPT_MODE_PAGEABLE | MPT_MODE_DUPLEX)) > 1 ||
        v[2] > 63) {
      std::fclose(f);
      return fail(MPT_EINVAL, "mpt_tune_load: %s line %u is not a tuner entry", path, lineno);
    }
    TuneEntry e;
    e.layout = (uint32_t)v[3];
    e.us = v[4];
    e.npaths = (uint32_t)((n - 5) / 5);
    for (uint32_t p = 0; p < e.npaths; ++p) {
      const double* q = v + 5 + 5 * p;
      e.paths[p] = mpt_path_spec{(uint32_t)q[0], (uint32_t)q[1], (uint64_t)q[2], (uint32_t)q[3], (uint32_t)q[4]};
    }
    mpt_plan_t probe = nullptr;
    if (mpt_plan(nullptr, 1ull << (uint32_t)v[2], (uint32_t)v[0], e.paths, e.npaths, 16, MPT_LAYOUT_CONTIG, &probe) !=
        MPT_OK) {
      std::fclose(f);
      return fail(MPT_EINVAL, "mpt_tune_load: %s line %u holds an invalid path set", path, lineno);
    }
    mpt_plan_destroy(probe);
    c->tuned[tune_key((uint32_t)v[0], (uint32_t)v[1], (uint32_t)v[2])] = e;
  }
  std::fclose(f);
  return MPT_OK;
}

mpt_status mpt_tune_get(mpt_ctx_t c, uint32_t dir, uint64_t nbytes, uint32_t mode, mpt_path_spec* out,
                        uint32_t* out_n, double* out_us) {
  if (!c || !out || !out_n) return fail(MPT_EINVAL, "mpt_tune_get: NULL argument");
  auto it = c->tuned.find(tune_key(dir, mode, size_bucket(nbytes)));
  if (it == c->tuned.end()) return fail(MPT_EAGAIN, "mpt_tune_get: no tuned entry for this bucket");
  std::memcpy(out, it->second.paths, it->second.npaths * sizeof(mpt_path_spec));
  *out_n = it->second.npaths;
  if (out_us) *out_us = it->second.us;
  return MPT_OK;
}

}  // extern "C"
