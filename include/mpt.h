/*
 * mpt.h -- C ABI of the single-GPU multi-path transfer library.
 *
 * Problem statement (Sec. 4.3, Algorithm 1 "CreateGraph"): move N bytes from a source
 * buffer to a destination buffer by splitting the message over a set of transfer paths
 * (the horizontal split, one share per path), cutting each path's part into chunks (the
 * vertical split) and running every path at the same time; the whole workflow is built
 * once as a CUDA graph, cached, and replayed (Sec. 4.2 "CUDA Graph Engine" / "CUDA Graph
 * Cache", Algorithm 1 "LaunchGraph").  On one GPU the paths are:
 *
 *   MPT_PATH_CE  copy-engine DMA, one memcpy per chunk (Algorithm 2 "PeerToPeerCopy");
 *   MPT_PATH_SM  a copy kernel driven by the SMs (device-to-device only);
 *   MPT_PATH_HS  a two-hop staged route, hop two of a chunk after its hop one
 *                (Algorithm 2 "StageHostCopy"): device-to-device goes through pinned
 *                host slots (three by default, MPT_STAGE_SLOTS = 2..4; the paper double
 *                buffers); host-to-device and device-to-host go through a device stage,
 *                chained by device-side chunk-ready flags, or with MPT_HS_HOST_THREADS
 *                through pinned slots filled and drained by host threads;
 *   MPT_PATH_ZC  a zero-copy kernel that reads or writes mapped pinned host memory
 *                directly over the host link (host-to-device and device-to-host only).
 *
 * Conventions for every call:
 *   - Every function returns mpt_status; nothing aborts or exits.  On failure
 *     mpt_last_error() returns a thread-local message describing the last error.
 *   - "stream" arguments are cudaStream_t values passed as void* (NULL = the legacy
 *     default stream).  Device pointers are CUDA device addresses; "host" buffers must be
 *     page-locked (cudaHostAlloc / cudaHostRegister / mpt_host_alloc) so that copy engines
 *     and kernels can reach them -- except on devices that reach pageable memory directly
 *     (cudaDevAttrPageableMemoryAccess, e.g. GB300 with its coherent Grace host), where
 *     plans made only of zero-copy paths, batches and mpt_sm_copy also accept ordinary
 *     pageable host memory.  Plans made only of zero-copy and host-thread staging paths
 *     (MPT_HS_HOST_THREADS) accept it on any device where those paths can run.
 *   - A context (mpt_ctx_t) owns its streams, events, staging buffers, device status
 *     word, graph cache and tuner cache.  One host thread per context.
 *   - Asynchronous calls only enqueue work; results are valid after the stream the work
 *     joined has been synchronised.  Device-side waits are bounded: a wait that gives up
 *     records MPT_ETIMEDOUT in the context's status word (mpt_ctx_status) instead of
 *     hanging the GPU.
 */
#ifndef MPT_H
#define MPT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define MPT_API __attribute__((visibility("default")))
#else
#define MPT_API
#endif

#define MPT_SHARE_ONE 65536u          /* shares are parts of 65536 */
#define MPT_MAX_PATHS 8u
#define MPT_MAX_ALIGN 4096u
#define MPT_MAX_CHUNKS (1u << 20)     /* chunks per plan */

typedef enum {
  MPT_OK = 0,
  MPT_EINVAL = 1,     /* invalid argument or plan */
  MPT_ENOMEM = 2,     /* allocation failed */
  MPT_EAGAIN = 3,     /* admission refused (staging budget or slots), retry later */
  MPT_ETIMEDOUT = 4,  /* a bounded device-side or host-side wait gave up */
  MPT_ENOTSUP = 5,    /* not supported on this device */
  MPT_ECUDA = 6       /* a CUDA runtime call failed; see mpt_last_error() */
} mpt_status;

typedef enum { MPT_D2D = 0, MPT_H2D = 1, MPT_D2H = 2 } mpt_dir;
typedef enum { MPT_PATH_CE = 1, MPT_PATH_SM = 2, MPT_PATH_HS = 4, MPT_PATH_ZC = 8 } mpt_path_kind;
typedef enum { MPT_LAYOUT_CONTIG = 0, MPT_LAYOUT_INTERLEAVE = 1 } mpt_layout;
/* OR into mpt_plan's layout to ask the tuner for its eager-mode (non-graph) choice. */
#define MPT_PLAN_EAGER 0x100u
/* OR into mpt_plan's layout (H2D/D2H) when the host buffer is ordinary pageable memory: the
 * tuner then chooses among the paths that accept it -- the zero-copy kernel (devices that
 * reach pageable memory) and host-thread staging -- from entries tuned with
 * MPT_MODE_PAGEABLE, else zero-copy alone (host-thread staging where the device cannot reach
 * pageable memory). */
#define MPT_PLAN_PAGEABLE 0x200u
/* OR into mpt_plan's layout (H2D/D2H, page-locked host memory) when the opposite direction
 * of the host link carries traffic at the same time (the paper's bidirectional test,
 * Sec. 5.3): the tuner's entry measured in both directions at once (MPT_MODE_DUPLEX), else
 * one copy-engine chunk -- one copy-engine node per direction kept both directions at their
 * shared rate (171.6 GB/s each on GB300) where plans tuned one direction at a time, with
 * zero-copy shares, reached 147-157 GB/s. */
#define MPT_PLAN_DUPLEX 0x400u
typedef enum { MPT_MODE_GRAPH = 0, MPT_MODE_EAGER = 1 } mpt_mode;
/* OR into mpt_tune's / mpt_tune_get's mode: tune (look up) the pageable-host-memory choice. */
#define MPT_MODE_PAGEABLE 0x10u
/* OR into mpt_tune's / mpt_tune_get's mode (H2D/D2H, page-locked): tune (look up) the choice
 * for a link whose other direction carries equal traffic (the paper's bidirectional test):
 * each candidate path set runs in both directions at once, the same set mirrored on another
 * stream, and is timed until both finish. */
#define MPT_MODE_DUPLEX 0x20u

/* mpt_path_spec.flags for SM-kernel paths: which copy kernel variant to run. */
#define MPT_SM_VEC128 0u   /* 128-bit vector loads/stores, grid-stride over 64 KiB tiles */
#define MPT_SM_BULK 1u     /* cp.async.bulk global->shared->global ring per CTA */
/* Ring configurations of the MPT_SM_BULK kernel, chosen per context by MPT_BULK_CONFIG=i
 * (0 <= i < MPT_BULK_CONFIGS, default 3) at context creation.  Stages x stage bytes, CTAs per SM:
 * 0: 4 x 48 KiB, 1; 1: as 0 with an L2 evict-first policy; 2: 3 x 64 KiB, 1; 3: 2 x 48 KiB, 2;
 * 4: as 3 with an L2 evict-first policy; 5: 3 x 32 KiB, 2; 6: 8 x 24 KiB, 1. */
#define MPT_BULK_CONFIGS 7u
#define MPT_SM_TILE8K 2u   /* VEC128 over 8 KiB tiles: a message of a few MiB reaches every SM
                              (BULK takes precedence when both are set) */
/* mpt_path_spec.flags for MPT_PATH_HS in H2D/D2H: host-thread staging.  The host side of each
 * chunk is a CPU copy, by the context's pool of host threads, between the caller's host buffer
 * and a page-locked slot; the device side is a copy-engine hop between the slot and device
 * memory (two slots, hop two of a chunk after its hop one, a slot refilled after its previous
 * hop two; Algorithm 2 StageHostCopy with a CPU hop).  The host buffer may be pageable.
 * MPT_HOST_THREADS at context creation sets the pool's worker count (default min(8, cores/2)
 * - 1; the thread that runs the CUDA host function copies a part as well).  Graphs with
 * this path are not retargeted in place (mpt_graph_rebind: ENOTSUP), and the eager engine
 * refuses it inside a stream capture (each eager launch owns its CPU-hop jobs). */
#define MPT_HS_HOST_THREADS 1u

/* One path of a plan.
 *   kind         one mpt_path_kind; allowed kinds per direction:
 *                D2D {CE, SM, HS}, H2D {CE, ZC, HS}, D2H {CE, ZC, HS}.
 *   share        this path's part of the message in 1/65536 units (> 0; all sum to 65536).
 *   chunk_bytes  C_p, chunk size of the vertical split; a positive multiple of the
 *                alignment, or 0 to let the context's tuner choose (needs a context).
 *   ctas         grid size for kernel lanes (0 = library default); ignored by CE.
 *   flags        kernel variant (MPT_SM_*), 0 otherwise. */
typedef struct {
  uint32_t kind;
  uint32_t share;
  uint64_t chunk_bytes;
  uint32_t ctas;
  uint32_t flags;
} mpt_path_spec;

/* One chunk of a plan: bytes [offset, offset+bytes) of the message go down path
 * path_index as that path's chunk number chunk_index. */
typedef struct {
  uint64_t offset;
  uint64_t bytes;
  uint32_t path_index;
  uint32_t chunk_index;
} mpt_chunk;

/* One transfer of a batch: copy `bytes` bytes from src to dst in direction dir. */
typedef struct {
  const void* src;
  void* dst;
  uint64_t bytes;
  uint32_t dir;
  uint32_t flags;
} mpt_xfer;

/* Graph lifecycle figures of a captured transfer (Sec. 5.5: creation, construction,
 * instantiation; launch is timed by the caller). */
typedef struct {
  uint32_t nodes;          /* graph nodes, every kind */
  uint32_t memcpy_nodes;
  uint32_t kernel_nodes;
  uint32_t memset_nodes;
  double create_us;        /* cudaGraphCreate */
  double construct_us;     /* adding nodes and edges */
  double instantiate_us;   /* cudaGraphInstantiate */
  uint64_t staging_bytes;  /* staging memory this graph owns */
  double update_us;        /* last in-place retarget (mpt_graph_rebind or a capture that reused it) */
  uint32_t rebinds;        /* in-place retargets so far */
  uint32_t mode;           /* 0: a CUDA graph; 1: prepared for direct issue (mpt_prepare) */
  uint32_t host_nodes;     /* CPU hops of host-thread staging */
} mpt_graph_info;

/* Cost model of one path kind: per-chunk issue latency and bandwidth (the staged path's
 * two hops have separate bandwidths; other kinds ignore beta2_Bps). */
typedef struct {
  uint64_t alpha_ps;
  uint64_t beta_Bps;
  uint64_t beta2_Bps;
} mpt_path_model;

/* Cost model of a plan (stated by this library; the paper tunes offline by exhaustive
 * search over link bandwidths and latencies, Sec. 4.4, without printing a model):
 * launch latency, HBM bandwidth, host-link bandwidth per direction, and one
 * mpt_path_model per path kind.  Bandwidths in bytes/s, times in picoseconds. */
typedef struct {
  uint64_t launch_ps;
  uint64_t hbm_Bps;
  uint64_t link_h2d_Bps;
  uint64_t link_d2h_Bps;
  mpt_path_model ce, sm, hs, zc;
} mpt_model;

typedef struct mpt_ctx_s* mpt_ctx_t;
typedef struct mpt_plan_s* mpt_plan_t;
typedef struct mpt_graph_s* mpt_graph_t;
typedef struct mpt_batch_s* mpt_batch_t;

/* ---- library and context ------------------------------------------------------- */

/* Version string; static storage. */
MPT_API const char* mpt_version(void);

/* Message of the last failed call on this thread; static thread-local storage. */
MPT_API const char* mpt_last_error(void);

/* Create a context on `device` (makes it current).  tune_file: path of a tuner cache to
 * load (JSON written by mpt_tune_save), or NULL for $MPT_TUNE_FILE, else the offline-tuned
 * defaults shipped next to the library as tuned/<device name>.jsonl when they exist
 * (MPT_TUNE_DEFAULTS=0 skips them).  Sec. 4.2 "Base Module": probes the
 * device and creates streams, events and the status word.  Errors: EINVAL (bad device),
 * ECUDA, ENOMEM. */
MPT_API mpt_status mpt_ctx_create(int device, const char* tune_file, mpt_ctx_t* out);

/* Destroy a context and everything it owns (cached graphs included).  Waits for the
 * device to go idle first.  Handles created from it become invalid. */
MPT_API mpt_status mpt_ctx_destroy(mpt_ctx_t ctx);

/* What the context found when it probed its device (Sec. 4.2 "Base Module"). */
typedef struct {
  char name[96];
  int32_t device;
  int32_t sms;               /* streaming multiprocessors */
  int32_t copy_engines;      /* asynchronous copy engines */
  int32_t pageable_access;   /* 1: kernels reach pageable host memory (coherent host) */
  uint64_t l2_bytes;
  uint64_t memory_bytes;
} mpt_device_info;

MPT_API mpt_status mpt_ctx_info(mpt_ctx_t ctx, mpt_device_info* out);

/* Lane timers: while enabled (or MPT_TRACE_LANES=1 at context creation), every multi-path
 * eager launch (mpt_launch_eager, or mpt_launch of an eager-prepared handle that forks onto
 * lanes; not inside a stream capture) records CUDA events at the start and end of each
 * path's lane.  mpt_lane_times waits for the last such launch and writes each path's
 * duration in milliseconds to out_ms[path index] (-1 for paths it did not time); *n gets
 * one past the last timed path.  Shows how evenly a split balances its paths. */
MPT_API mpt_status mpt_trace_lanes(mpt_ctx_t ctx, uint32_t enable);
MPT_API mpt_status mpt_lane_times(mpt_ctx_t ctx, float* out_ms, uint32_t cap, uint32_t* n);

/* Read the context's device status word (blocking: synchronises the device), return it
 * (MPT_OK or the first recorded MPT_ETIMEDOUT) and reset it to MPT_OK.  `site` (nullable)
 * receives an implementation-defined code of the wait that gave up. */
MPT_API mpt_status mpt_ctx_status(mpt_ctx_t ctx, uint32_t* site);

/* Set the wait limit of the staged host-to-device path's device-side flag waits (hop two
 * waiting for a chunk's hop one, Algorithm 2 StageHostCopy) for every graph of this context,
 * captured before or after the call: the limit lives in device memory and each wait reads it
 * when it starts.  ns = 0 restores the default (2 s); ns above 10 s is refused.  A wait that
 * runs out records MPT_ETIMEDOUT (mpt_ctx_status) and its CTA stops; the transfer's
 * destination is then incomplete, and the next replay of the same graph starts from zeroed
 * flags.  Synchronises the device first.  Errors: EINVAL, ECUDA. */
MPT_API mpt_status mpt_ctx_set_wait_limit(mpt_ctx_t ctx, uint64_t ns);

/* ---- planning (Sec. 4.3 horizontal + vertical split; Algorithm 1) ----------------- */

/* Build the chunk plan for an `nbytes` message in direction `dir` over `npaths` paths.
 * ctx may be NULL when every path has an explicit chunk size.  paths == NULL asks the
 * tuner for the whole path set (Sec. 4.4): the environment (MPT_PATHS=ce,sm,hs,zc,
 * MPT_SHARES=w0,w1.., MPT_CHUNK_BYTES=C or MPT_CHUNKS=k per path, MPT_CTAS,
 * MPT_SM_VARIANT=vec|bulk) when MPT_PATHS is set, else the context's tuned entry for
 * this (direction, mode, log2 size) bucket, else the cost model's best split; chunk_bytes
 * 0 on a listed path asks the same sources for that path's chunk size.  Without
 * MPT_PATHS these need a context.  layout | MPT_PLAN_EAGER selects the eager-mode
 * choices.  align: chunk offsets are
 * multiples of it (power of two <= 4096; 16 is the library's default).  layout:
 * CONTIG gives each path one contiguous region in path order; INTERLEAVE deals chunks
 * round robin (Sec. 4.3, the text after Algorithm 2).  Horizontal split: path p < P-1
 * gets floor_A(floor(N*share_p/65536)) bytes, the last path the remainder; every chunk
 * but a path's last has chunk_bytes bytes.  The plan is owned by the caller
 * (mpt_plan_destroy).  Errors: EINVAL for a bad argument, a kind that cannot carry
 * `dir`, shares not summing to 65536, a zero share, a chunk size that is not a positive
 * multiple of `align`, or more than MPT_MAX_CHUNKS chunks. */
MPT_API mpt_status mpt_plan(mpt_ctx_t ctx, uint64_t nbytes, uint32_t dir, const mpt_path_spec* paths,
                    uint32_t npaths, uint32_t align, uint32_t layout, mpt_plan_t* out);

/* Copy up to `cap` chunks, sorted by (path_index, chunk_index), into `out` (nullable when
 * cap == 0) and store the total count in *n. */
MPT_API mpt_status mpt_plan_chunks(mpt_plan_t plan, mpt_chunk* out, size_t cap, size_t* n);

/* Copy the plan's resolved path specs (chunk sizes and CTA counts filled in) into `out`
 * (capacity `cap`) and store the path count in *n. */
MPT_API mpt_status mpt_plan_paths(mpt_plan_t plan, mpt_path_spec* out, uint32_t cap, uint32_t* n);

MPT_API mpt_status mpt_plan_destroy(mpt_plan_t plan);

/* ---- graph capture, cache and launch (Algorithm 1 CreateGraph / LaunchGraph) ------ */

/* Return the executable graph that moves plan's message from src to dst, building,
 * instantiating and caching it on a miss (key: src, dst, N, direction, plan hash;
 * fixed-capacity LRU, capacity MPT_GRAPH_CACHE, default 64; Sec. 4.2 "CUDA Graph
 * Cache").  On a miss, a cached graph of the same plan that only the cache holds is
 * retargeted in place (cudaGraphExecUpdate) instead of instantiating a new one, the graph
 * update Sec. 6 leaves as future work; MPT_GRAPH_REBIND=0 disables this.  src/dst must match the plan's direction (device or page-locked host memory)
 * and must stay allocated while the graph can run: a graph is bound to its addresses.
 * *out is a new reference owned by the caller (mpt_graph_release); eviction from the
 * cache never invalidates a held reference.  Graphs with a staged path own their
 * staging memory.  Errors: EINVAL (pointer kind does not fit the direction, chunk of a
 * staged path above the stage size), ECUDA, ENOMEM. */
MPT_API mpt_status mpt_capture(mpt_ctx_t ctx, mpt_plan_t plan, void* dst, const void* src, mpt_graph_t* out);

/* Prepare a transfer for repeated launches with mpt_launch, as a graph (mode
 * MPT_PREPARE_GRAPH, exactly mpt_capture), for direct issue on the launching stream
 * (MPT_PREPARE_EAGER: the eager engine of mpt_launch_eager, with no fork/join at all when
 * the plan uses a single copy-engine or kernel path), or whichever of the two the
 * context's tuner measured faster for this direction and log2 size bucket
 * (MPT_PREPARE_AUTO; graph when either measurement is missing).  The paper finds graphs
 * help only above a few MB and tunes graph and non-graph execution separately (Sec. 4.4,
 * Sec. 5.3).  Release with mpt_graph_release; eager handles are not cached. */
typedef enum { MPT_PREPARE_GRAPH = 0, MPT_PREPARE_EAGER = 1, MPT_PREPARE_AUTO = 2 } mpt_prepare_mode;
MPT_API mpt_status mpt_prepare(mpt_ctx_t ctx, mpt_plan_t plan, void* dst, const void* src, uint32_t mode,
                               mpt_graph_t* out);

/* Launch a captured graph on `stream`: it starts after the work already queued on the
 * stream and later work on the stream waits for all of its chunks (Sec. 4.5 "Final
 * Synchronization").  Asynchronous.  Launches of one graph run one after another. */
MPT_API mpt_status mpt_launch(mpt_graph_t graph, void* stream);

/* Lifecycle figures of a captured graph. */
MPT_API mpt_status mpt_graph_get_info(mpt_graph_t graph, mpt_graph_info* out);

/* Retarget a captured graph at new addresses of the same sizes without re-instantiating
 * it: the node set is rebuilt for (dst, src) with the graph's own staging buffers and the
 * executable is updated in place.  `plan` must be the plan the graph was captured from.
 * Every holder of the handle sees the new addresses; its cache entry is re-keyed.  The
 * update applies to later launches.  Errors: EINVAL (other plan, wrong pointer kinds),
 * EAGAIN (another cached graph already serves those addresses), ENOTSUP (the runtime
 * cannot update in place, e.g. the SM kernel variant changes with the new alignment --
 * capture anew). */
MPT_API mpt_status mpt_graph_rebind(mpt_graph_t graph, mpt_plan_t plan, void* dst, const void* src);

/* Drop a graph reference obtained from mpt_capture. */
MPT_API mpt_status mpt_graph_release(mpt_graph_t graph);

/* Drop every cached graph whose source or destination range contains `ptr` (call before
 * freeing a buffer that cached graphs refer to); *n (nullable) gets the count. */
MPT_API mpt_status mpt_graph_evict(mpt_ctx_t ctx, const void* ptr, uint32_t* n);

/* Issue the same multi-path workflow without a graph (Sec. 4.3's static runtime
 * pipelining engine): fork from `stream` onto per-path lane streams, enqueue every chunk,
 * join back onto `stream`.  Asynchronous.  Eager transfers that use the same staged path
 * serialise on that path's lane (Sec. 4.5 "Contention Avoidance").  A plan with a single
 * copy-engine or kernel path is issued on `stream` itself, without fork or join; outside a
 * stream capture its copy kernels are launched with programmatic dependent launch, so that
 * their launch overlaps the end of a copy kernel before them on `stream` (they wait for its
 * completion before touching memory).  MPT_PDL=0 at context creation turns that off. */
MPT_API mpt_status mpt_launch_eager(mpt_ctx_t ctx, mpt_plan_t plan, void* dst, const void* src, void* stream);

/* ---- single kernels (the SM and zero-copy paths on their own) -------------------- */

/* Copy `nbytes` from src to dst with one launch of the SM copy kernel on `stream`.
 * Both pointers must be device-accessible (device memory, or mapped page-locked host
 * memory for the zero-copy direction).  variant: MPT_SM_VEC128, MPT_SM_BULK (the bulk
 * variant handles the 16-byte-aligned body with cp.async.bulk and the rest with plain
 * loads; it falls back to VEC128 when src and dst differ modulo 16) or MPT_SM_TILE8K
 * (device memory only; ignored for the zero-copy direction).  ctas: grid size,
 * 0 = default.  ctx supplies the status word for bounded waits.  Errors: EINVAL. */
MPT_API mpt_status mpt_sm_copy(mpt_ctx_t ctx, void* dst, const void* src, uint64_t nbytes, uint32_t variant,
                       uint32_t ctas, void* stream);

/* Digest of a device-accessible byte range, computed on the GPU on `stream`, waited for,
 * and stored in *out: H = mix64(N) + sum_i mix64(w_i XOR i*0x9E3779B97F4A7C15) mod 2^64,
 * w_i the little-endian 8-byte words of the range zero-padded, mix64 the splitmix64
 * output finaliser.  Blocking. */
MPT_API mpt_status mpt_hash_device(mpt_ctx_t ctx, const void* ptr, uint64_t nbytes, void* stream, uint64_t* out);

/* ---- cost model and split search (tuner building blocks; host only, no GPU) -------- */

/* Modelled time in picoseconds of `npaths` paths of kinds `kinds` carrying bytes[p] each
 * in chunks of `chunk` bytes, direction `dir`:
 *   T_p  = alpha_p * ceil(b_p/C) + ceil(b_p * 1e12 / beta_p)
 *   T_HS = alpha * (ceil(b/C) + 1) + ceil(b*1e12/min(beta,beta2)) + ceil(min(C,b)*1e12/max(beta,beta2))
 *   T    = launch + max(max_p T_p, T_HBM, T_link_h2d, T_link_d2h)
 * where T_HBM and T_link count how often each payload byte crosses HBM (2 device-to-
 * device; 1 direct host transfer; 3 host transfer through a device stage) and the link
 * (once per crossing, per direction).  Integer arithmetic, ceilings as written.
 * Errors: EINVAL (zero bandwidth, kind not allowed for `dir`, chunk 0). */
MPT_API mpt_status mpt_model_time(const mpt_model* m, uint32_t dir, const uint32_t* kinds, const uint64_t* bytes,
                                  uint32_t npaths, uint64_t chunk, uint64_t* out_ps);

/* Best split of an `nbytes` message over 1..4 paths under the model: paths 0..P-2 take
 * multiples of `step` bytes (step = align for nbytes <= 4096 -- an exhaustive search --
 * else floor_align(nbytes/64), i.e. 1/64 shares), the last path the remainder; chunk
 * sizes align*2^k <= max(nbytes, align) shared by all paths.  Ties: lowest time, fewest
 * non-empty paths, lexicographically largest split, largest chunk.  out_bytes receives
 * npaths byte counts. */
MPT_API mpt_status mpt_model_optimize(const mpt_model* m, uint64_t nbytes, uint32_t dir, const uint32_t* kinds,
                                      uint32_t npaths, uint32_t align, uint64_t* out_bytes, uint64_t* out_chunk,
                                      uint64_t* out_ps);

/* ---- autotuner (Sec. 4.4: tuned paths/chunks, separately for graph and eager mode) ---- */

/* Measure candidate path sets for an `nbytes` message in direction `dir` and execution
 * mode `mode` (MPT_MODE_GRAPH or MPT_MODE_EAGER) on this context's GPU -- single copy
 * engine paths with 1..8 chunks, the SM kernel (vec128/bulk, several CTA counts), the
 * zero-copy kernel, copy engine + kernel splits at several shares and chunk counts (a
 * winning split is then refined in 1/64 steps of its share), the staged path -- each the
 * median of `reps` timed runs (0 = default), every run starting
 * with a cold L2 full of dirty lines (a 256 MiB write first, as after the kernel that
 * produced the data; a message of at most 64 MiB is timed as the mean of 8 back-to-back
 * launches after it, each on its own buffer region -- the regime of a stream of messages,
 * where launch costs overlap).  The three fastest candidates and the fastest single-path
 * candidate of each path kind are then timed again in interleaved rounds (one run of each
 * per round, at least 5 rounds), so that drift between candidates timed far apart cannot
 * decide the choice; the lowest median of those rounds is stored for the message's log2
 * size bucket.  With mode | MPT_MODE_PAGEABLE
 * (H2D/D2H) the host buffer is ordinary pageable memory and the candidates are the paths
 * that accept it: the zero-copy kernel, host-thread staging (MPT_HS_HOST_THREADS) and their
 * splits; the entry serves mpt_plan(..., MPT_PLAN_PAGEABLE).  Blocking;
 * allocates scratch buffers of `nbytes` (kept by the context).  MPT_TUNE_VERBOSE=1 prints
 * every candidate's timing to stderr.  out (capacity 4, nullable),
 * out_n and out_us (nullable) receive the winner.  Errors: EINVAL, ECUDA, ENOMEM. */
MPT_API mpt_status mpt_tune(mpt_ctx_t ctx, uint32_t dir, uint64_t nbytes, uint32_t mode, uint32_t reps,
                            mpt_path_spec* out, uint32_t* out_n, double* out_us);

/* Write every tuned entry as JSON lines {"dir","mode","bucket","layout","us","paths":
 * [[kind, share, chunk_bytes, ctas, flags], ...]}. */
MPT_API mpt_status mpt_tune_save(mpt_ctx_t ctx, const char* path);

/* Load entries written by mpt_tune_save (also done by mpt_ctx_create for its tune_file
 * argument or $MPT_TUNE_FILE).  Errors: EINVAL for an unreadable file or invalid entry. */
MPT_API mpt_status mpt_tune_load(mpt_ctx_t ctx, const char* path);

/* The tuned entry for the bucket of `nbytes` (EAGAIN when there is none). */
MPT_API mpt_status mpt_tune_get(mpt_ctx_t ctx, uint32_t dir, uint64_t nbytes, uint32_t mode, mpt_path_spec* out,
                                uint32_t* out_n, double* out_us);

/* ---- batched transfers (persistent descriptor-table kernel, replayed graph) ----------- */

/* Size the context's batch ring: `slots` batches in flight at once (default 4), up to
 * `max_xfers` transfers per batch (default 4096), `ctas` CTAs of the batch kernel
 * (default 3 x SMs) and `tile_bytes` per work item (default 256 KiB; >= 4096, multiple of
 * 16).  tile_bytes is the largest tile: a batch whose kernel-moved bytes give each CTA less
 * than one tile is cut into the power of two at or above its bytes per CTA (at least
 * 32 KiB), so that a short batch spreads over the grid.  0 keeps a default.  Waits for the
 * device; fails with EAGAIN while a batch is held.  The ring is built on first use with
 * defaults when this is never called. */
MPT_API mpt_status mpt_batch_configure(mpt_ctx_t ctx, uint32_t slots, uint32_t max_xfers, uint32_t ctas,
                                       uint32_t tile_bytes);

/* DMA lanes of the batch (the batch kernel plus copy-engine lanes): per direction (D2D, H2D,
 * D2H) `lanes` copy-engine lanes, each taking up to `items_per_lane` entries of at least
 * `min_bytes` per batch, largest first to the least-loaded lane of the entry's direction;
 * the kernel moves everything else.  Entries with a pageable host side stay with the
 * kernel.  Each lane entry completes individually (time stamp and host flag, as for kernel
 * entries).  lanes = 0 turns the lanes off (the default unless MPT_BATCH_DMA_LANES,
 * MPT_BATCH_DMA_ITEMS and MPT_BATCH_DMA_MIN set them).  Rebuilds the batch ring like
 * mpt_batch_configure.  Errors: EINVAL (lanes > 8, items outside 1..64, min_bytes < 16),
 * EAGAIN (a batch is held), ECUDA. */
MPT_API mpt_status mpt_batch_configure_dma(mpt_ctx_t ctx, uint32_t lanes, uint32_t items_per_lane,
                                           uint64_t min_bytes);

/* Batch autotuner (CTA count, tile size and DMA lanes chosen by measurement).  Runs the representative
 * batch `xfers` (n entries; their destinations are written) `reps` times (0 = 3) under each
 * candidate setting -- kernel CTAs in {1, 2, 3} x SMs, tile bytes in {64, 128, 256, 512,
 * 1024} KiB, DMA lanes off or 2 per direction for entries of at least 4 MiB -- and keeps the
 * best: objective MPT_BATCH_TUNE_TIME the shortest median batch, MPT_BATCH_TUNE_P99 the
 * lowest median p99 entry completion time (device clock, from the kernel's start).  The
 * chosen setting is applied to the context (as mpt_batch_configure and
 * mpt_batch_configure_dma would) and written to *out (nullable).  Blocking.  Errors: EINVAL,
 * EAGAIN (a batch is held), ECUDA. */
#define MPT_BATCH_TUNE_TIME 0u
#define MPT_BATCH_TUNE_P99 1u
typedef struct {
  uint32_t ctas;           /* kernel CTAs */
  uint32_t tile_bytes;
  uint32_t dma_lanes;      /* per direction, 0 = kernel alone */
  uint32_t dma_items;
  uint64_t dma_min_bytes;
  double batch_us;         /* median batch time of the chosen setting */
  double p99_us;           /* median p99 entry completion of the chosen setting */
  uint32_t candidates;     /* settings measured */
  uint32_t reserved;
} mpt_batch_tuning;

MPT_API mpt_status mpt_batch_tune(mpt_ctx_t ctx, const mpt_xfer* xfers, size_t n, uint32_t objective, uint32_t reps,
                                  void* stream, mpt_batch_tuning* out);

/* Register an arena (this GPU's memory or page-locked host memory) so that batch
 * descriptors inside it are classified without per-pointer runtime queries.  The caller
 * keeps ownership; the arena must stay allocated while registered. */
MPT_API mpt_status mpt_batch_register(mpt_ctx_t ctx, const void* base, uint64_t bytes);

/* Move n transfers in one launch of the persistent batch kernel, as one replay of a slot's
 * graph on `stream` (windowed transfers, Sec. 5.3: many messages in flight, one launch).
 * The kernel's CTAs claim fixed-size tiles of the transfers through two cursors: tiles of
 * transfers with a host side (over the host link) and device-to-device tiles.  The first
 * 32 CTAs (MPT_BATCH_LINK_CTAS=k: k) start on the former and move to device tiles when they
 * run out; the others take device tiles only.  32 CTAs hold the link at its rate, and
 * keeping no more of its traffic in flight keeps short what other batches' transfers,
 * table copies and completion flags wait behind on the link (MPT_BATCH_SPLIT=0: one cursor
 * over every tile in table order, every CTA on it).
 * Each xfer: D2D (device -> device), H2D (page-locked host -> device, read over the host
 * link by the kernel) or D2H (device -> page-locked host).  Destinations must not overlap
 * (Sec. 4.5: each transfer owns its region).  The descriptor table is copied into the
 * slot, so `xfers` may be reused on return; the replay copies only the table's used bytes
 * to the device (a few hundred for a short batch) and the kernel resets its own counters,
 * so a one-transfer batch is one small copy and one kernel.  *out is owned by the caller until
 * mpt_batch_release, which frees the slot.  Errors: EINVAL (bad descriptor, overlapping
 * destinations, n outside 1..max_xfers), EAGAIN (every slot held), ECUDA. */
MPT_API mpt_status mpt_batch_submit(mpt_ctx_t ctx, const mpt_xfer* xfers, size_t n, void* stream, mpt_batch_t* out);

/* Non-blocking: number of the batch's transfers that have completed (their destination
 * bytes are written and visible), read from page-locked per-transfer flags the kernel
 * raises as each transfer's last tile finishes; flags (nullable, n bytes) gets 1/0 per
 * transfer. */
MPT_API mpt_status mpt_batch_poll(mpt_batch_t batch, size_t* done, uint8_t* flags);

/* Wait up to timeout_ns for the whole batch (bounded host wait).  ETIMEDOUT when it is
 * still running -- the batch keeps running and may be waited for again. */
MPT_API mpt_status mpt_batch_wait(mpt_batch_t batch, uint64_t timeout_ns);

/* Completion time of every transfer in nanoseconds after the batch kernel started (device
 * global timer); waits for the batch.  out_ns has n entries. */
MPT_API mpt_status mpt_batch_times(mpt_batch_t batch, uint64_t* out_ns);

/* Wait up to timeout_ns for the whole batch while watching its per-transfer completion
 * flags from the host, and write to out_ns[i] (n entries) the mpt_now_ns time at which
 * transfer i's flag was first seen, minus t0_ns (0 if it was seen before t0_ns).  With t0_ns
 * taken just before mpt_batch_submit, out_ns is each transfer's latency from submission as
 * a host thread observes it -- the same origin and observer as mpt_copy_each, so that
 * batched and per-transfer copies compare like for like (Sec. 5.3's windowed bandwidth: many
 * messages in flight).  The flags are scanned in a spin loop, so resolution is a few
 * microseconds.  Errors: EINVAL, ETIMEDOUT (still running, or the batch ended with a
 * transfer unflagged), ECUDA. */
MPT_API mpt_status mpt_batch_watch(mpt_batch_t batch, uint64_t t0_ns, uint64_t* out_ns, uint64_t timeout_ns);

/* Release the handle and its slot. */
MPT_API mpt_status mpt_batch_release(mpt_batch_t batch);

/* The per-transfer baseline of a batch: every transfer as its own cudaMemcpyAsync, in table
 * order, transfer i on streams[xfers[i].dir] (three entries: D2D, H2D, D2H; entries may
 * repeat, NULL is the legacy default stream).  Giving each direction its own stream keeps
 * device-to-device copies from queueing behind copies limited by the host link (Sec. 4.5,
 * contention avoidance).  out_ns NULL: asynchronous, returns once every copy is enqueued.
 * out_ns non-NULL (n entries): after enqueueing, waits up to timeout_ns and writes each
 * transfer's completion time as seen by this host thread (its completion event polled in a
 * spin loop), in nanoseconds after the call was entered.  The copies use cudaMemcpyDefault,
 * so pointer kinds are not checked beyond NULL and the direction code.  Errors: EINVAL,
 * ETIMEDOUT, ECUDA. */
MPT_API mpt_status mpt_copy_each(mpt_ctx_t ctx, const mpt_xfer* xfers, size_t n, void* const* streams, uint64_t* out_ns,
                                 uint64_t timeout_ns);

/* ---- serving loop (continuous batching over the batch ring) ------------------------ */

typedef struct mpt_server_s* mpt_server_t;

typedef struct {
  uint64_t staging_budget_bytes;  /* admission limit on bytes in flight (0 = $MPT_STAGING_BUDGET, else 8 GiB) */
  uint32_t max_batch;             /* transfers per batch (0 = the slot capacity) */
  uint32_t max_inflight_batches;  /* batches on the GPU at once (0 = every slot) */
  uint32_t streams;               /* streams batches are launched on (0 = one per batch in flight;
                                     1 = every batch in submission order) */
  uint32_t batch_ctas;            /* batch kernel CTAs (0 = one per SM, so that several batch
                                     kernels share the SMs); the ring keeps it after the server stops */
} mpt_serve_config;

/* One finished request: its tag, the arrival time the caller gave, when it was admitted
 * into a batch and when its completion flag was seen (mpt_now_ns clock), its size, and
 * MPT_OK or the error that refused it. */
typedef struct {
  uint64_t tag;
  uint64_t arrival_ns;
  uint64_t admit_ns;
  uint64_t complete_ns;
  uint64_t bytes;
  uint32_t status;
  uint32_t reserved;
} mpt_completion;

/* Counters of a running server.  max_pending_completions: the most finished requests
 * that waited at once for mpt_serve_poll; max_turn_ns: the worker's longest single turn
 * (harvest + admit + launch), which bounds how late it can notice a finished batch or a
 * free slot, and the longest of each of those three phases; max_waiting: the longest
 * admission queue seen; max_batch_ns: the longest batch, from its launch to the release of
 * its slot, with its request count and bytes. */
typedef struct {
  uint64_t submitted, completed, batches, inflight_bytes, max_inflight_bytes, rejected;
  uint64_t max_pending_completions, max_turn_ns, max_waiting;
  uint64_t max_batch_ns, max_batch_reqs, max_batch_bytes;
  uint64_t max_harvest_ns, max_admit_ns, max_launch_ns;
} mpt_serve_stats_t;

/* The clock of mpt_serve_submit / mpt_completion (steady, nanoseconds). */
MPT_API uint64_t mpt_now_ns(void);

/* Start a serving loop on `ctx` (cfg nullable = defaults).  A worker thread owns the
 * context until mpt_serve_stop: do not use the context from other threads meanwhile.  It
 * admits waiting requests oldest first while the bytes in flight stay within the budget (a
 * request larger than the whole budget runs alone), packs them into the next batch, and
 * launches it as soon as a batch slot is free, so requests arriving while earlier batches
 * run overlap with them on the device.  Each request completes individually when the
 * batch kernel raises its flag.  By default each batch in flight gets a stream of its own
 * and the batch kernel one CTA per SM, so a batch of short requests runs beside an earlier
 * batch with a long one instead of behind it (on GB300 at 50k requests/s, 2 s: p50 from
 * submit 28 us against 130 us in order on one stream with three CTAs per SM, p99 277 us
 * against 1.31 ms); requests in flight are then unordered and must not share destination
 * bytes.  An idle worker spins on the arrival flag for MPT_SERVE_SPIN_US microseconds
 * (default 2000; 0 = block at once) after its last work before it blocks, so a request
 * after a short gap is not delayed by a thread wake-up (one core busy while the server is
 * active). */
MPT_API mpt_status mpt_serve_start(mpt_ctx_t ctx, const mpt_serve_config* cfg, mpt_server_t* out);

/* Enqueue one request (thread-safe).  arrival_ns: the request's scheduled arrival on the
 * mpt_now_ns clock (0 = now); latency is measured from it.  The same rules as
 * mpt_batch_submit apply to the transfer.  A request that breaks them on its own (direction,
 * NULL pointer, memory kinds) is refused alone when it is admitted: its completion carries
 * the error and the requests around it are unaffected.  The caller must keep destinations
 * of requests in flight from overlapping one another or any source in flight; a batch
 * that breaks this is refused as a whole. */
MPT_API mpt_status mpt_serve_submit(mpt_server_t server, const mpt_xfer* xfer, uint64_t tag, uint64_t arrival_ns);

/* Move up to `cap` finished requests, oldest first, into `out` (thread-safe); *n gets the
 * count.  Costs O(*n) under the server's lock whatever the backlog, so a client that falls
 * behind does not slow the worker or the submitters. */
MPT_API mpt_status mpt_serve_poll(mpt_server_t server, mpt_completion* out, size_t cap, size_t* n);

MPT_API mpt_status mpt_serve_stats(mpt_server_t server, mpt_serve_stats_t* out);

/* Zero the high-water marks of mpt_serve_stats (every max_* field), leaving the running
 * counts (submitted, completed, batches, inflight_bytes, rejected) as they are: for example
 * after a warm-up, or at the start of each monitoring interval.  A worker update that races
 * with the reset may survive it.  Errors: EINVAL (NULL server). */
MPT_API mpt_status mpt_serve_reset_stats(mpt_server_t server);

/* Replay a request trace: submit xfers[i] (tag tags[i]) at its scheduled time due_ns[i]
 * (mpt_now_ns clock, non-decreasing), spinning between arrivals, from the calling thread --
 * a load generator that keeps the schedule to about a microsecond where a slower client
 * would add its own lateness to every latency.  Returns once every request is submitted;
 * completions arrive through mpt_serve_poll as usual (poll from another thread meanwhile).
 * late_ns (nullable, n entries) receives each submission's delay past its scheduled time.
 * Errors: EINVAL (NULL arrays, decreasing times), those of mpt_serve_submit. */
MPT_API mpt_status mpt_serve_replay(mpt_server_t server, const mpt_xfer* xfers, const uint64_t* tags,
                                    const uint64_t* due_ns, size_t n, uint64_t* late_ns);

/* Finish every request already submitted, stop the worker and free the server.
 * Completions not yet polled are dropped. */
MPT_API mpt_status mpt_serve_stop(mpt_server_t server);

/* ---- compute for the compute-plus-communication demonstration ------------------------ */

/* One Jacobi sweep over a subdomain (the paper's application study, Sec. 5.4: subdomains in
 * a ring exchange boundary rows with both neighbours), so that stencil kernels and
 * multi-path halo exchanges can be captured together into one graph.  in/out: (rows + 2)
 * x cols fp32 row-major device arrays, rows 0 and rows+1 the halos.  Interior points:
 * out[r][c] = ((in[r-1][c] + in[r+1][c]) + (in[r][c-1] + in[r][c+1])) * 0.25, each operation
 * rounded to fp32 in that order; columns 0 and cols-1 copied; out's halo rows untouched.
 * Asynchronous on `stream` (legal inside a stream capture).  Errors: EINVAL. */
MPT_API mpt_status mpt_demo_jacobi_step(const float* in, float* out, uint32_t rows, uint64_t cols, void* stream);

/* ---- failure detection self-test ---------------------------------------------------- */

/* Launch the staged path's consumer kernel on one chunk whose ready flag nothing raises,
 * with a device-side wait limit of timeout_ns (<= 10 s), and return the context status it
 * leaves: MPT_ETIMEDOUT with *site (nullable) = the wait's site code, and the GPU usable.
 * Demonstrates that bounded device waits report instead of hanging. */
MPT_API mpt_status mpt_selftest_flag_timeout(mpt_ctx_t ctx, uint64_t timeout_ns, uint32_t* site);

/* ---- digests without allocation ------------------------------------------------------ */

/* Digests (the mpt_hash_device function) of n device byte ranges, computed on `stream`,
 * waited for, and written to out[0..n).  The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory when they need it (a caller-owned
 * memory budget or allocator that must not be bypassed, or code that must not trigger the
 * device synchronisation cudaMalloc/cudaFree can cause).  It allocates nothing: the
 * per-range accumulators live in a static device array of MPT_NOALLOC_MAX_RANGES entries
 * (8 KiB) that every GPU loading the library holds until the process exits.  No context
 * is needed; it runs on the current device.  The first call on a device looks up the
 * array's device address once; make that first call before any stream capture.  Every
 * call shares the array, so calls whose work overlaps on the GPU (different streams or
 * host threads at the same time) race and must be serialised by the caller.  Errors:
 * EINVAL (n above the maximum, NULL argument), ECUDA. */
#define MPT_NOALLOC_MAX_RANGES 1024u
MPT_API mpt_status mpt_hash_ranges_noalloc(const void* const* ptrs, const uint64_t* nbytes, uint32_t n, void* stream,
                                           uint64_t* out);

/* ---- page-locked host memory ---------------------------------------------------- */

/* Allocate `nbytes` of page-locked, device-mapped host memory for staging and zero-copy
 * transfers (Sec. 4.3's host-staged path moves chunks through such buffers).  ctx (nullable):
 * its device is made current first.  *host receives the host address; dev_alias (nullable)
 * receives the address device code uses for it (cudaHostGetDevicePointer; with unified
 * addressing, as on GB300, the same value).  Copy engines and the zero-copy kernel accept
 * either.  The caller owns the buffer: free it with mpt_host_free (with the same ctx, which
 * records the buffer).  Errors: EINVAL (NULL host), ENOMEM, ECUDA (no device address). */
MPT_API mpt_status mpt_host_alloc(mpt_ctx_t ctx, uint64_t nbytes, void** host, void** dev_alias);

/* Free a buffer from mpt_host_alloc.  With the context it was allocated with, every graph that
 * context has cached on the buffer (source or destination range overlapping it) is dropped
 * from the cache first, as mpt_graph_evict would: a cached graph bound to freed page-locked
 * memory must never be launched or retargeted.  Handles the caller still holds stay valid
 * objects but must not be launched again.  ctx may be NULL (no eviction). */
MPT_API mpt_status mpt_host_free(mpt_ctx_t ctx, void* ptr);

/* Host-memory bandwidth with CPU threads alone: the memory every host-link path (copy
 * engines, zero-copy kernel, staged paths; Sec. 4.3, Sec. 5.2) reads or writes on the host
 * side.  `threads` host threads each stream over their contiguous part of [ptr, ptr+nbytes),
 * `reps` times: op 0 reads every 8-byte word, op 1 writes every word, op 2 copies the first
 * half of the buffer into the second.  *out_gbs gets the best rep's host-memory traffic in
 * GB/s (bytes read plus bytes written).  Blocking; host only, no GPU work.  Errors: EINVAL
 * (NULL argument, op above 2, threads outside 1..1024, a buffer under 4 KiB per thread). */
MPT_API mpt_status mpt_host_bandwidth(void* ptr, uint64_t nbytes, uint32_t threads, uint32_t op, uint32_t reps,
                                      double* out_gbs);

#ifdef __cplusplus
}
#endif

#endif /* MPT_H */
