// Serving loop: continuous batching of transfer requests over the batch ring.
//
// Requests arrive on any host thread (mpt_serve_submit).  One worker thread owns the
// context while the server runs and repeats:
//   1. harvest: read the host-mapped completion flags of every batch in flight and
//      complete each finished request individually (its completion time, the bytes it
//      held against the budget returned); a batch whose requests are all done and whose
//      graph has finished gives its slot back;
//   2. admit: move waiting requests, oldest first, into the batch under construction while
//      the bytes in flight stay within the staging budget and the batch has room;
//   3. launch: when a slot is free, submit the batch under construction (one graph replay
//      of the persistent batch kernel).  Requests that arrive while earlier batches are
//      still on the GPU wait only for a slot, not for those batches to finish, so their
//      work overlaps on the device -- the windowed, many-in-flight regime where the paper
//      finds graphs pay off (Sec. 5.3).
// Batches in flight run on streams of their own (by default) and the batch kernel takes one
// CTA per SM, so several batch kernels share the SMs: a batch of short requests is not held
// behind an earlier batch with a long one.
// Latency is measured from the scheduled arrival time the caller passes, so a late caller
// does not hide queueing delay.  An idle worker spins on the arrival flag for a while before
// it blocks, so a request arriving after a short gap does not wait for a thread wake-up.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "ctx.h"

namespace mpt {
namespace {

// An idle worker spins this long after its last work before it blocks (MPT_SERVE_SPIN_US;
// 0 blocks at once).  Two milliseconds cover most gaps between requests at 1k/s and above.
constexpr uint64_t kDefaultSpinUs = 2000;

uint64_t steady_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  mpt_xfer x;
  uint64_t tag, arrival_ns, admit_ns;
};

// One launched batch, for the optional batch log (MPT_SERVE_BATCH_LOG).
struct BatchRecord {
  uint64_t launch_ns, done_ns, reqs, bytes, bytes_dir[3];
  uint32_t stream;
  float gpu_ms;  // device time of the replay (timing events), -1 if unknown
  uint64_t cta_spread_ns;  // first to last CTA start of the batch kernel
};

struct InFlight {
  mpt_batch_t batch;
  uint32_t stream;                // index into the server's streams
  uint64_t launch_ns = 0, bytes = 0;
  uint64_t bytes_dir[3] = {0, 0, 0};
  std::vector<Request> reqs;
  std::vector<uint8_t> flags;     // last poll: 1 = finished
  std::vector<uint8_t> reported;  // completion already handed out
  size_t ndone = 0;
};

}  // namespace
}  // namespace mpt

struct mpt_server_s {
  mpt_ctx_t ctx = nullptr;
  mpt_serve_config cfg{};
  std::vector<cudaStream_t> streams;
  std::thread worker;
  // Two locks, so that submitters and the polling client never wait for each other:
  // mu guards incoming, stop and error (submit side), out_mu the completions (poll side).
  std::mutex mu;
  std::condition_variable cv;
  std::deque<mpt::Request> incoming;
  // set (under mu) when incoming gains a request or a stop is asked for: a busy worker locks
  // mu only then, so its turns do not contend with submitters for the lock
  std::atomic<bool> wake{false};
  std::atomic<bool> failed{false};  // error != MPT_OK, readable without mu
  std::mutex out_mu;
  std::deque<mpt_completion> completions;  // popped from the front: O(1) per entry
  std::atomic<size_t> pending{0};          // completions.size(): an empty poll takes no lock
  bool stop = false;
  mpt_status error = MPT_OK;
  std::string error_msg;
  std::atomic<uint64_t> submitted{0}, completed{0}, batches{0}, inflight_bytes{0}, max_inflight_bytes{0};
  std::atomic<uint64_t> rejected{0};
  std::atomic<uint64_t> max_pending{0}, max_turn_ns{0}, max_waiting{0};
  std::atomic<uint64_t> max_batch_ns{0}, max_batch_reqs{0}, max_batch_bytes{0};  // the longest batch
  std::atomic<uint64_t> max_harvest_ns{0}, max_admit_ns{0}, max_launch_ns{0};    // worker turn phases
  bool shortest_first = false;            // order each batch by size before launching it
  uint64_t spin_ns = 0;                   // MPT_SERVE_SPIN_US: idle spin before blocking
  std::string batch_log;                  // MPT_SERVE_BATCH_LOG: CSV written at stop
  // worker-owned until the worker exits; a deque, since a vector's doubling would copy
  // millions of records inside one worker turn
  std::deque<mpt::BatchRecord> records;
};

namespace mpt {
namespace {

void record_error(mpt_server_s* s, mpt_status st) {
  std::lock_guard<std::mutex> g(s->mu);
  if (s->error == MPT_OK) {
    s->error = st;
    s->error_msg = mpt_last_error();
    s->failed.store(true, std::memory_order_release);
  }
}

void serve_loop(mpt_server_s* s) {
  cudaSetDevice(s->ctx->device);
  std::deque<Request> waiting;
  std::vector<InFlight> flight;
  std::vector<Request> building;
  uint64_t budget_used = 0;
  std::vector<mpt_xfer> xs;
  std::vector<mpt_completion> done_local;
  std::vector<uint8_t> stream_busy(s->streams.size(), 0);  // a stream per batch in flight
  std::deque<Request> arrived;
  bool stopping = false;
  uint64_t last_busy = steady_ns();
  while (true) {
    const bool idle = waiting.empty() && flight.empty() && building.empty();
    if (!idle) last_busy = steady_ns();
    // an idle worker watches the arrival flag for spin_ns after its last work before it
    // blocks: waking a blocked thread costs several microseconds per request
    if (idle && s->spin_ns)
      while (!s->wake.load(std::memory_order_acquire) && steady_ns() - last_busy < s->spin_ns) {
      }
    if (idle || s->wake.load(std::memory_order_acquire)) {
      std::unique_lock<std::mutex> lk(s->mu);
      if (idle && s->incoming.empty() && !s->stop) s->cv.wait_for(lk, std::chrono::microseconds(200));
      arrived.swap(s->incoming);  // O(1) under the lock
      s->wake.store(false, std::memory_order_relaxed);
      stopping = s->stop;
    }
    for (const Request& r : arrived) waiting.push_back(r);
    arrived.clear();
    const uint64_t turn0 = steady_ns();
    if (waiting.size() > s->max_waiting) s->max_waiting = waiting.size();
    // 1. harvest
    done_local.clear();
    for (size_t i = 0; i < flight.size();) {
      InFlight& f = flight[i];
      size_t n = 0;
      if (mpt_batch_poll(f.batch, &n, f.flags.data()) != MPT_OK) {
        record_error(s, MPT_ECUDA);
        return;
      }
      if (n != f.ndone) {
        const uint64_t now = steady_ns();
        for (size_t k = 0; k < f.reqs.size(); ++k) {
          if (!f.flags[k] || f.reported[k]) continue;
          f.reported[k] = 1;
          const Request& r = f.reqs[k];
          done_local.push_back(mpt_completion{r.tag, r.arrival_ns, r.admit_ns, now, r.x.bytes, MPT_OK, 0});
          budget_used -= r.x.bytes;
        }
        f.ndone = n;
      }
      if (f.ndone == f.reqs.size() && mpt_batch_wait(f.batch, 0) == MPT_OK) {
        const uint64_t t_done = steady_ns();
        const uint64_t took = t_done - f.launch_ns;
        if (!s->batch_log.empty())
          s->records.push_back(BatchRecord{f.launch_ns, t_done, f.reqs.size(), f.bytes,
                                           {f.bytes_dir[0], f.bytes_dir[1], f.bytes_dir[2]}, f.stream,
                                           batch_gpu_ms(f.batch), batch_cta_spread_ns(f.batch)});
        if (took > s->max_batch_ns) {
          s->max_batch_ns = took;
          s->max_batch_reqs = f.reqs.size();
          s->max_batch_bytes = f.bytes;
        }
        mpt_batch_release(f.batch);
        stream_busy[f.stream] = 0;
        flight[i] = std::move(flight.back());
        flight.pop_back();
      } else {
        ++i;
      }
    }
    const uint64_t turn1 = steady_ns();
    // 2. admit, oldest first, within the budget and the batch capacity
    const uint64_t budget = s->cfg.staging_budget_bytes;
    while (!waiting.empty() && building.size() < s->cfg.max_batch) {
      const Request& r = waiting.front();
      int ks, kd;
      const mpt_status bad = batch_check_xfer(s->ctx, r.x, &ks, &kd);
      if (bad != MPT_OK) {  // refused on its own, before it can share a batch with others
        const uint64_t now = steady_ns();
        done_local.push_back(mpt_completion{r.tag, r.arrival_ns, now, now, r.x.bytes, (uint32_t)bad, 0});
        s->rejected++;
        waiting.pop_front();
        continue;
      }
      const bool alone = budget_used == 0 && building.empty();
      if (budget_used + r.x.bytes > budget && !alone) break;  // an oversized request goes alone
      Request q = r;
      q.admit_ns = steady_ns();
      budget_used += q.x.bytes;
      building.push_back(q);
      waiting.pop_front();
    }
    s->inflight_bytes = budget_used;
    if (budget_used > s->max_inflight_bytes) s->max_inflight_bytes = budget_used;
    const uint64_t turn2 = steady_ns();
    // 3. launch when a slot is free
    // one stream: batches run in submission order; several: each batch in flight has its own
    uint32_t si = 0;
    if (s->streams.size() > 1) {
      while (si < stream_busy.size() && stream_busy[si]) ++si;
    }
    bool launched = false;
    if (!building.empty() && flight.size() < s->cfg.max_inflight_batches && si < s->streams.size()) {
      if (s->shortest_first)  // tiles go out in descriptor order: short requests first
        std::stable_sort(building.begin(), building.end(),
                         [](const Request& a, const Request& b) { return a.x.bytes < b.x.bytes; });
      xs.resize(building.size());
      for (size_t k = 0; k < building.size(); ++k) xs[k] = building[k].x;
      mpt_batch_t b = nullptr;
      const mpt_status st = mpt_batch_submit(s->ctx, xs.data(), xs.size(), s->streams[si], &b);
      if (st == MPT_OK) {
        launched = true;
        if (s->streams.size() > 1) stream_busy[si] = 1;
        InFlight f;
        f.batch = b;
        f.stream = si;
        f.launch_ns = steady_ns();
        for (const Request& r : building) {
          f.bytes += r.x.bytes;
          f.bytes_dir[r.x.dir] += r.x.bytes;
        }
        f.reqs = std::move(building);
        f.flags.assign(f.reqs.size(), 0);
        f.reported.assign(f.reqs.size(), 0);
        flight.push_back(std::move(f));
        building.clear();
        s->batches++;
      } else if (st != MPT_EAGAIN) {
        // the batch as a whole was refused (requests in it overlap one another, which the
        // caller must not allow): complete them with the error, keep serving
        const uint64_t now = steady_ns();
        for (const Request& r : building) {
          done_local.push_back(mpt_completion{r.tag, r.arrival_ns, r.admit_ns, now, r.x.bytes, (uint32_t)st, 0});
          budget_used -= r.x.bytes;
        }
        s->rejected += building.size();
        building.clear();
      }
    }
    if (!done_local.empty()) {
      std::lock_guard<std::mutex> g(s->out_mu);
      s->completions.insert(s->completions.end(), done_local.begin(), done_local.end());
      s->pending.store(s->completions.size(), std::memory_order_release);
      s->completed += done_local.size();
      if (s->completions.size() > s->max_pending) s->max_pending = s->completions.size();
    }
    const uint64_t turn3 = steady_ns();
    if (turn3 - turn0 > s->max_turn_ns) s->max_turn_ns = turn3 - turn0;
    if (turn1 - turn0 > s->max_harvest_ns) s->max_harvest_ns = turn1 - turn0;
    if (turn2 - turn1 > s->max_admit_ns) s->max_admit_ns = turn2 - turn1;
    if (turn3 - turn2 > s->max_launch_ns) s->max_launch_ns = turn3 - turn2;
    if (stopping && waiting.empty() && building.empty() && flight.empty()) {
      std::lock_guard<std::mutex> g(s->mu);
      if (s->incoming.empty()) return;
    }
    if (!flight.empty() && !launched) std::this_thread::yield();
  }
}

}  // namespace
}  // namespace mpt

using namespace mpt;

extern "C" {

uint64_t mpt_now_ns(void) { return steady_ns(); }

mpt_status mpt_serve_start(mpt_ctx_t ctx, const mpt_serve_config* cfg, mpt_server_t* out) {
  if (!ctx || !out) return fail(MPT_EINVAL, "mpt_serve_start: NULL argument");
  *out = nullptr;
  for (auto& sl : ctx->slots)
    if (sl.held) return fail(MPT_EAGAIN, "mpt_serve_start: batches of this context are still held");
  const uint32_t want_ctas = cfg && cfg->batch_ctas ? cfg->batch_ctas : (uint32_t)ctx->sms;
  if (want_ctas != ctx->batch_ctas) {
    mpt_status st = mpt_batch_configure(ctx, ctx->batch_slots, ctx->batch_max_xfers, want_ctas, ctx->batch_tile);
    if (st != MPT_OK) return st;
  }
  mpt_status st = batch_setup(ctx);
  if (st != MPT_OK) return st;
  mpt_server_s* s = new mpt_server_s;
  s->ctx = ctx;
  mpt_serve_config c = cfg ? *cfg : mpt_serve_config{};
  if (c.staging_budget_bytes == 0) {
    const char* v = std::getenv("MPT_STAGING_BUDGET");
    c.staging_budget_bytes = (v && *v) ? std::strtoull(v, nullptr, 0) : 0;
    if (c.staging_budget_bytes == 0) c.staging_budget_bytes = 8ull << 30;
  }
  if (c.max_batch == 0 || c.max_batch > ctx->slots[0].max_xfers) c.max_batch = ctx->slots[0].max_xfers;
  if (c.max_inflight_batches == 0 || c.max_inflight_batches > ctx->slots.size())
    c.max_inflight_batches = (uint32_t)ctx->slots.size();
  if (c.streams == 0 || c.streams > c.max_inflight_batches) c.streams = c.max_inflight_batches;
  c.batch_ctas = want_ctas;
  s->cfg = c;
  if (const char* log = std::getenv("MPT_SERVE_BATCH_LOG")) s->batch_log = log;
  if (const char* o = std::getenv("MPT_SERVE_ORDER")) s->shortest_first = std::strcmp(o, "size") == 0;
  {
    const char* v = std::getenv("MPT_SERVE_SPIN_US");
    s->spin_ns = ((v && *v) ? std::strtoull(v, nullptr, 0) : kDefaultSpinUs) * 1000ull;
  }
  ctx->batch_timing = !s->batch_log.empty();
  if (cudaSetDevice(ctx->device) != cudaSuccess) {
    delete s;
    return fail(MPT_ECUDA, "mpt_serve_start: device");
  }
  s->streams.assign(c.streams, nullptr);
  for (auto& cs : s->streams)
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      for (auto& x : s->streams)
        if (x) cudaStreamDestroy(x);
      delete s;
      return fail(MPT_ECUDA, "mpt_serve_start: stream");
    }
  s->worker = std::thread(serve_loop, s);
  *out = s;
  return MPT_OK;
}

mpt_status mpt_serve_submit(mpt_server_t s, const mpt_xfer* x, uint64_t tag, uint64_t arrival_ns) {
  if (!s || !x) return fail(MPT_EINVAL, "mpt_serve_submit: NULL argument");
  if (x->dir > MPT_D2H) return fail(MPT_EINVAL, "mpt_serve_submit: direction %u", x->dir);
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return fail(MPT_EINVAL, "mpt_serve_submit: server is stopping");
    if (s->error != MPT_OK) return fail(s->error, "mpt_serve_submit: server failed: %s", s->error_msg.c_str());
    s->incoming.push_back(Request{*x, tag, arrival_ns ? arrival_ns : steady_ns(), 0});
    s->wake.store(true, std::memory_order_release);
  }
  s->submitted++;
  s->cv.notify_one();
  return MPT_OK;
}

mpt_status mpt_serve_replay(mpt_server_t s, const mpt_xfer* xfers, const uint64_t* tags, const uint64_t* due_ns,
                            size_t n, uint64_t* late_ns) {
  if (!s || (n > 0 && (!xfers || !tags || !due_ns))) return fail(MPT_EINVAL, "mpt_serve_replay: NULL argument");
  for (size_t i = 1; i < n; ++i)
    if (due_ns[i] < due_ns[i - 1]) return fail(MPT_EINVAL, "mpt_serve_replay: times decrease at %zu", i);
  for (size_t i = 0; i < n; ++i) {
    uint64_t now = steady_ns();
    while (now < due_ns[i]) {
      // spin through the last 50 us, sleep-yield before that
      if (due_ns[i] - now > 50000) std::this_thread::yield();
      now = steady_ns();
    }
    mpt_status st = mpt_serve_submit(s, &xfers[i], tags[i], due_ns[i]);
    if (late_ns) late_ns[i] = steady_ns() - due_ns[i];
    if (st != MPT_OK) return st;
  }
  return MPT_OK;
}

mpt_status mpt_serve_poll(mpt_server_t s, mpt_completion* out, size_t cap, size_t* n) {
  if (!s || !n || (cap && !out)) return fail(MPT_EINVAL, "mpt_serve_poll: NULL argument");
  *n = 0;
  if (cap && s->pending.load(std::memory_order_acquire) != 0) {
    std::lock_guard<std::mutex> g(s->out_mu);
    const size_t k = std::min(cap, s->completions.size());
    std::copy(s->completions.begin(), s->completions.begin() + k, out);
    s->completions.erase(s->completions.begin(), s->completions.begin() + k);
    s->pending.store(s->completions.size(), std::memory_order_relaxed);
    *n = k;
  }
  if (s->failed.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> g(s->mu);
    return fail(s->error, "mpt_serve_poll: server failed: %s", s->error_msg.c_str());
  }
  return MPT_OK;
}

mpt_status mpt_serve_stats(mpt_server_t s, mpt_serve_stats_t* out) {
  if (!s || !out) return fail(MPT_EINVAL, "mpt_serve_stats: NULL argument");
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->batches = s->batches;
  out->inflight_bytes = s->inflight_bytes;
  out->max_inflight_bytes = s->max_inflight_bytes;
  out->rejected = s->rejected;
  out->max_pending_completions = s->max_pending;
  out->max_turn_ns = s->max_turn_ns;
  out->max_waiting = s->max_waiting;
  out->max_batch_ns = s->max_batch_ns;
  out->max_batch_reqs = s->max_batch_reqs;
  out->max_batch_bytes = s->max_batch_bytes;
  out->max_harvest_ns = s->max_harvest_ns;
  out->max_admit_ns = s->max_admit_ns;
  out->max_launch_ns = s->max_launch_ns;
  return MPT_OK;
}

mpt_status mpt_serve_reset_stats(mpt_server_t s) {
  if (!s) return fail(MPT_EINVAL, "mpt_serve_reset_stats: NULL server");
  for (std::atomic<uint64_t>* m : {&s->max_inflight_bytes, &s->max_pending, &s->max_turn_ns, &s->max_waiting,
                                   &s->max_batch_ns, &s->max_batch_reqs, &s->max_batch_bytes, &s->max_harvest_ns,
                                   &s->max_admit_ns, &s->max_launch_ns})
    m->store(0);
  return MPT_OK;
}

mpt_status mpt_serve_stop(mpt_server_t s) {
  if (!s) return MPT_OK;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    s->wake.store(true, std::memory_order_release);
  }
  s->cv.notify_one();
  if (s->worker.joinable()) s->worker.join();
  mpt_status st = s->error;
  if (st != MPT_OK) fail(st, "mpt_serve_stop: server failed: %s", s->error_msg.c_str());
  s->ctx->batch_timing = false;
  // completions not yet polled are dropped with the server
  for (cudaStream_t cs : s->streams) {
    cudaStreamSynchronize(cs);
    cudaStreamDestroy(cs);
  }
  if (!s->batch_log.empty()) {  // one line per batch, launch order not guaranteed
    if (FILE* f = std::fopen(s->batch_log.c_str(), "w")) {
      std::fprintf(f, "launch_ns,done_ns,requests,bytes,d2d_bytes,h2d_bytes,d2h_bytes,stream,gpu_ms,cta_spread_us\n");
      for (const BatchRecord& r : s->records)
        std::fprintf(f, "%llu,%llu,%llu,%llu,%llu,%llu,%llu,%u,%.4f,%.1f\n", (unsigned long long)r.launch_ns,
                     (unsigned long long)r.done_ns, (unsigned long long)r.reqs, (unsigned long long)r.bytes,
                     (unsigned long long)r.bytes_dir[0], (unsigned long long)r.bytes_dir[1],
                     (unsigned long long)r.bytes_dir[2], r.stream, r.gpu_ms, r.cta_spread_ns / 1e3);
      std::fclose(f);
    }
  }
  delete s;
  return st;
}

}  // extern "C"
