// server.cu -- corr_server_*: a served X-engine.  Blocks of several arrays
// arrive one by one from the host, are staged into an HBM arena, integrated
// into each array's resident accumulators and returned as visibilities once
// an integration is complete.
//
// The paper's pipeline (Sec. 2.3) runs hashpipe threads around ring buffers:
// a network thread fills block slots, the GPU thread correlates them, an
// output thread ships integrations.  Here one worker thread owns every CUDA
// call and drives
//   copy       host block -> arena slot (H2D), one stream,
//   compute    one stream per array: its pushes and dumps (the CMAC and dump
//              kernels), in the order its accumulators need,
//   out        visibilities -> pinned host result buffer (D2H), one stream,
// so copies of later blocks overlap the correlation of earlier ones, and the
// CMAC launches of different arrays run concurrently on the device: a block
// admitted while another array's work is on the GPU starts as soon as SMs
// free up instead of queueing behind it (continuous batching of the arrays'
// requests).
//
// Blocks carry (array, sequence number).  Integration k of an array holds
// sequence numbers [k L, (k + 1) L).  Sums are exact integers, so blocks may
// be integrated in any order:
//   - a block of a later integration (up to `window` integrations ahead) is
//     staged and held until its integration is current;
//   - a block that would open an integration `window` or more ahead closes
//     the current one, which then completes with the blocks it holds (the
//     others were dropped upstream);
//   - a duplicate of an accepted block and a block of a closed integration
//     are discarded and counted.
// A result names the blocks it integrated (a bit mask), so a receiver can
// tell complete from partial integrations.
//
// Admission: a block enters only when its bytes fit in the arena (first fit,
// coalescing free list) -- blocks wait in arrival order while it is full, so
// the HBM budget bounds what is in flight.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <thread>
#include <vector>

#include "corr.h"
#include "trace.h"

namespace {

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return CORR_OK;
  if (e == cudaErrorMemoryAllocation) return CORR_ENOMEM;
  return CORR_ECUDA;
}

// First-fit allocator over [0, size) with a coalescing free list.
class Arena {
 public:
  explicit Arena(size_t size) : size_(size) {
    if (size) free_[0] = size;
  }
  // Returns the offset, or SIZE_MAX when no free range is large enough.
  size_t alloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > bytes) free_[off + bytes] = len - bytes;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return off;
    }
    return SIZE_MAX;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    used_ -= bytes;
    auto next = free_.lower_bound(off);
    if (next != free_.end() && next->first == off + bytes) {
      bytes += next->second;
      next = free_.erase(next);
    }
    if (next != free_.begin()) {
      auto prev = std::prev(next);
      if (prev->first + prev->second == off) {
        prev->second += bytes;
        return;
      }
    }
    free_[off] = bytes;
  }
  size_t peak() const { return peak_; }

 private:
  size_t size_, used_ = 0, peak_ = 0;
  std::map<size_t, size_t> free_;  // offset -> length
};

enum BlkState { kWaiting, kCopying, kCopied, kPushed };

struct Blk {
  long long seq;
  const uint8_t *h;
  double t_arr;
  BlkState state;
  size_t off;
  cudaEvent_t copied, pushed;
};

struct Integ {
  std::map<long long, Blk> blocks;  // by sequence number
  bool closed = false;
};

struct Array {
  corr_array_desc d;
  size_t block_bytes, vis_elems;
  corr_ctx *ctx = nullptr;
  cudaStream_t s_compute = nullptr;  // this array's pushes and dumps
  bool stream_shared = false;        // s_compute belongs to array 0
  int64_t *d_vis = nullptr, *h_vis = nullptr;
  long long cur = 0;                 // current integration
  long long closed_below = 0;        // every integration below this is closed
  std::map<long long, Integ> integ;  // current and held later integrations
  // dump in flight (at most one per array); result_held is guarded by the
  // server's mutex (the caller releases it)
  bool dumping = false, result_held = false;
  cudaEvent_t dumped = nullptr;
  corr_result pending;
  std::vector<double> pending_arrivals;
};

struct Req {
  int array;
  long long seq;
  const uint8_t *h;
  double t_arr;
};

double percentile(std::vector<double> v, double p) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double x = p * (double)(v.size() - 1);
  const size_t i = (size_t)x;
  const double f = x - (double)i;
  return i + 1 < v.size() ? v[i] * (1.0 - f) + v[i + 1] * f : v[i];
}

}  // namespace

struct corr_server {
  std::vector<Array> arrays;
  int window = 2;
  int device = 0;
  bool dry = false;
  uint8_t *d_arena = nullptr;
  Arena *arena = nullptr;
  cudaStream_t s_copy = nullptr, s_out = nullptr;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_results;
  std::deque<Req> inbox;
  std::deque<Req> waiting;  // accepted, not yet admitted into the arena (worker only)
  std::deque<corr_result> results;
  bool stop = false, flush_req = false;
  int error = CORR_OK;
  // events of finished blocks, reused by later blocks (worker only), so that
  // the steady state creates no events
  std::vector<cudaEvent_t> ev_pool;
  bool take_event(cudaEvent_t *e) {
    if (!ev_pool.empty()) {
      *e = ev_pool.back();
      ev_pool.pop_back();
      return true;
    }
    return cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  }
  void give_event(cudaEvent_t &e) {
    if (e) ev_pool.push_back(e);
    e = nullptr;
  }
  // statistics
  long long n_submitted = 0, n_integrated = 0, n_dup = 0, n_late = 0, n_incomplete = 0,
            n_integrations = 0;
  std::vector<double> latencies;
  // worker-side helpers
  void run();
  bool step();
  void classify(const Req &r);
  void close_upto(Array &a, long long k);
  bool admit();
  bool progress(int ai);
};

namespace {

Blk *find_blk(Array &a, long long seq) {
  const long long k = seq / a.d.blocks_per_integration;
  auto it = a.integ.find(k);
  if (it == a.integ.end()) return nullptr;
  auto b = it->second.blocks.find(seq);
  return b == it->second.blocks.end() ? nullptr : &b->second;
}

}  // namespace

// Closes every integration of `a` below k (they complete with what they
// hold; those that hold nothing are skipped).
void corr_server::close_upto(Array &a, long long k) {
  for (auto &kv : a.integ)
    if (kv.first < k) kv.second.closed = true;
  a.closed_below = std::max(a.closed_below, k);
}

void corr_server::classify(const Req &r) {
  Array &a = arrays[r.array];
  const int L = a.d.blocks_per_integration;
  const long long k = r.seq / L;
  if (r.seq < 0 || k < a.cur || (k < a.closed_below && !a.integ.count(k))) {
    ++n_late;  // a finished integration, or one closed before this block came
    return;
  }
  auto it = a.integ.find(k);
  if (it != a.integ.end() && (it->second.closed || it->second.blocks.count(r.seq))) {
    if (it->second.blocks.count(r.seq)) ++n_dup;
    else ++n_late;
    return;
  }
  if (k >= a.cur + window) close_upto(a, k - window + 1);
  Integ &in = a.integ[k];
  Blk b;
  std::memset(&b, 0, sizeof(b));
  b.seq = r.seq;
  b.h = r.h;
  b.t_arr = r.t_arr;
  b.state = kWaiting;
  in.blocks[r.seq] = b;
  waiting.push_back(r);
}

// Moves waiting blocks into the arena in arrival order; returns whether any moved.
bool corr_server::admit() {
  bool moved = false;
  while (!waiting.empty()) {
    const Req r = waiting.front();
    Array &a = arrays[r.array];
    Blk *b = find_blk(a, r.seq);
    if (!b || b->state != kWaiting) {
      waiting.pop_front();
      continue;
    }
    const size_t off = arena->alloc(a.block_bytes);
    if (off == SIZE_MAX) break;  // full: later blocks wait behind this one
    b->off = off;
    if (!dry) {
      CORR_TRACE("server_copy_block");
      if (!take_event(&b->copied) ||
          cudaMemcpyAsync(d_arena + off, b->h, a.block_bytes, cudaMemcpyHostToDevice, s_copy) !=
              cudaSuccess ||
          cudaEventRecord(b->copied, s_copy) != cudaSuccess) {
        error = CORR_ECUDA;
        return false;
      }
    }
    b->state = kCopying;
    waiting.pop_front();
    moved = true;
  }
  return moved;
}

// Pushes copied blocks of the current integration, frees slots of pushed
// blocks, dumps complete integrations and publishes finished dumps.
bool corr_server::progress(int ai) {
  Array &a = arrays[ai];
  bool moved = false;
  // a finished dump becomes a result
  if (a.dumping && (dry || cudaEventQuery(a.dumped) == cudaSuccess)) {
    a.dumping = false;
    const double t = now_ms();
    a.pending.t_done_ms = t;
    {
      std::lock_guard<std::mutex> lock(mu);
      a.result_held = true;
      for (double ta : a.pending_arrivals) latencies.push_back(t - ta);
      results.push_back(a.pending);
    }
    cv_results.notify_all();
    moved = true;
  }
  for (auto &kv : a.integ) {
    for (auto &bk : kv.second.blocks) {
      Blk &b = bk.second;
      if (b.state == kCopying && (dry || cudaEventQuery(b.copied) == cudaSuccess)) {
        b.state = kCopied;
        moved = true;
      }
      if (b.state == kPushed && b.off != SIZE_MAX &&
          (dry || cudaEventQuery(b.pushed) == cudaSuccess)) {
        arena->release(b.off, a.block_bytes);
        b.off = SIZE_MAX;
        moved = true;
      }
    }
  }
  auto it = a.integ.find(a.cur);
  if (it == a.integ.end()) return moved;
  Integ &in = it->second;
  const int L = a.d.blocks_per_integration;
  // push the current integration's copied blocks (nothing is pushed while
  // the previous integration's dump is still being read out of the
  // accumulators: stream order on the compute stream takes care of that)
  for (auto &bk : in.blocks) {
    Blk &b = bk.second;
    if (b.state != kCopied) continue;
    if (!dry) {
      CORR_TRACE("server_push_block");
      if (cudaStreamWaitEvent(a.s_compute, b.copied, 0) != cudaSuccess ||
          corr_push_block(a.ctx, d_arena + b.off, a.s_compute) != CORR_OK ||
          !take_event(&b.pushed) || cudaEventRecord(b.pushed, a.s_compute) != cudaSuccess) {
        error = CORR_ECUDA;
        return false;
      }
    }
    b.state = kPushed;
    moved = true;
  }
  int n_pushed = 0;
  bool all_pushed = true;
  for (auto &bk : in.blocks) {
    if (bk.second.state == kPushed) ++n_pushed;
    else all_pushed = false;
  }
  const bool complete = n_pushed == L || (in.closed && all_pushed);
  if (!complete || a.dumping) return moved;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (a.result_held) return moved;
  }
  // dump: visibilities to the pinned result buffer
  corr_result res;
  std::memset(&res, 0, sizeof(res));
  res.array = ai;
  res.integration = a.cur;
  res.n_blocks = n_pushed;
  res.t_first_arrival_ms = 1e300;
  res.t_last_arrival_ms = 0.0;
  a.pending_arrivals.clear();
  for (auto &bk : in.blocks) {
    const Blk &b = bk.second;
    res.block_mask |= 1ull << (b.seq - a.cur * L);
    res.t_first_arrival_ms = std::min(res.t_first_arrival_ms, b.t_arr);
    res.t_last_arrival_ms = std::max(res.t_last_arrival_ms, b.t_arr);
    a.pending_arrivals.push_back(b.t_arr);
  }
  res.vis = dry ? nullptr : a.h_vis;
  if (!dry) {
    CORR_TRACE("server_dump");
    if (corr_dump(a.ctx, a.d_vis, nullptr, a.s_compute) != CORR_OK ||
        cudaEventRecord(a.dumped, a.s_compute) != cudaSuccess ||
        cudaStreamWaitEvent(s_out, a.dumped, 0) != cudaSuccess ||
        cudaMemcpyAsync(a.h_vis, a.d_vis, a.vis_elems * sizeof(int64_t), cudaMemcpyDeviceToHost,
                        s_out) != cudaSuccess ||
        cudaEventRecord(a.dumped, s_out) != cudaSuccess) {
      error = CORR_ECUDA;
      return false;
    }
  }
  a.pending = res;
  a.dumping = true;
  {
    std::lock_guard<std::mutex> lock(mu);
    ++n_integrations;
    n_integrated += n_pushed;
    if (n_pushed < L) ++n_incomplete;
  }
  // the integration's blocks stay recorded until their slots are free
  in.closed = true;
  ++a.cur;
  return true;
}

bool corr_server::step() {
  bool moved = false;
  std::deque<Req> got;
  bool flush = false;
  {
    std::lock_guard<std::mutex> lock(mu);
    got.swap(inbox);
    flush = flush_req;
    flush_req = false;
  }
  for (const Req &r : got) classify(r);
  moved |= !got.empty();
  if (flush)
    for (Array &a : arrays) {
      long long top = a.cur;
      for (auto &kv : a.integ) top = std::max(top, kv.first + 1);
      close_upto(a, top);
      moved = true;
    }
  moved |= admit();
  for (int ai = 0; ai < (int)arrays.size(); ++ai) moved |= progress(ai);
  // forget integrations whose blocks are all pushed and whose slots are free
  for (Array &a : arrays)
    for (auto it = a.integ.begin(); it != a.integ.end();) {
      bool done = it->first < a.cur;
      for (auto &bk : it->second.blocks)
        if (bk.second.state != kPushed || bk.second.off != SIZE_MAX) done = false;
      if (done) {
        if (!dry)
          for (auto &bk : it->second.blocks) {
            give_event(bk.second.copied);
            give_event(bk.second.pushed);
          }
        it = a.integ.erase(it);
      } else {
        ++it;
      }
    }
  // skip past integrations that were closed while empty
  for (Array &a : arrays)
    while (a.cur < a.closed_below && a.integ.find(a.cur) == a.integ.end()) {
      ++a.cur;
      moved = true;
    }
  return moved;
}

void corr_server::run() {
  if (!dry && cudaSetDevice(device) != cudaSuccess) {
    std::lock_guard<std::mutex> lock(mu);
    error = CORR_ECUDA;
    cv_results.notify_all();
    return;
  }
  for (;;) {
    const bool moved = step();
    std::unique_lock<std::mutex> lock(mu);
    if (error != CORR_OK) {
      cv_results.notify_all();
      return;
    }
    if (stop) return;  // the destroyer synchronises the streams
    if (!moved && inbox.empty() && !flush_req)
      cv_work.wait_for(lock, std::chrono::microseconds(50));
  }
}

namespace {

void free_server(corr_server *s) {
  if (!s) return;
  if (s->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lock(s->mu);
      s->stop = true;
    }
    s->cv_work.notify_all();
    s->worker.join();
  }
  if (!s->dry) {
    if (s->s_copy) cudaStreamSynchronize(s->s_copy);
    for (Array &a : s->arrays)
      if (a.s_compute) cudaStreamSynchronize(a.s_compute);
    if (s->s_out) cudaStreamSynchronize(s->s_out);
    for (Array &a : s->arrays) {
      if (a.s_compute && !a.stream_shared) cudaStreamDestroy(a.s_compute);
      corr_destroy(a.ctx);
      cudaFree(a.d_vis);
      cudaFreeHost(a.h_vis);
      if (a.dumped) cudaEventDestroy(a.dumped);
      for (auto &kv : a.integ)
        for (auto &bk : kv.second.blocks) {
          if (bk.second.copied) cudaEventDestroy(bk.second.copied);
          if (bk.second.pushed) cudaEventDestroy(bk.second.pushed);
        }
    }
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
    cudaFree(s->d_arena);
    if (s->s_copy) cudaStreamDestroy(s->s_copy);
    if (s->s_out) cudaStreamDestroy(s->s_out);
  }
  delete s->arena;
  delete s;
}

}  // namespace

extern "C" {

int corr_server_create(int n_arrays, const corr_array_desc *desc, size_t arena_bytes, int window,
                       int flags, corr_server **out) {
  CORR_TRACE("corr_server_create");
  if (!out) return CORR_EINVAL;
  *out = nullptr;
  if (n_arrays <= 0 || !desc || window < 1 || (flags & ~CORR_SERVER_DRY)) return CORR_EINVAL;
  size_t largest = 0;
  for (int k = 0; k < n_arrays; ++k) {
    const corr_array_desc &d = desc[k];
    if (d.n_ant <= 0 || d.n_chan <= 0 || d.block_len <= 0 || (d.n_pol != 1 && d.n_pol != 2) ||
        d.block_len > CORR_MAX_BLOCK_LEN || (long long)d.n_ant * d.n_pol > CORR_MAX_INPUTS ||
        d.blocks_per_integration < 1 || d.blocks_per_integration > 64)
      return CORR_EINVAL;
    largest = std::max(largest, (size_t)d.n_chan * d.n_ant * d.n_pol * d.block_len);
  }
  if (arena_bytes < (largest + 255) / 256 * 256) return CORR_EINVAL;
  corr_server *s = new (std::nothrow) corr_server;
  if (!s) return CORR_ENOMEM;
  s->dry = (flags & CORR_SERVER_DRY) != 0;
  s->window = window;
  s->arena = new (std::nothrow) Arena(arena_bytes);
  if (!s->arena) {
    delete s;
    return CORR_ENOMEM;
  }
  s->arrays.resize(n_arrays);
  int rc = CORR_OK;
  for (int k = 0; k < n_arrays; ++k) {
    Array &a = s->arrays[k];
    a.d = desc[k];
    const long long n_in = (long long)a.d.n_ant * a.d.n_pol;
    a.block_bytes = (size_t)a.d.n_chan * n_in * a.d.block_len;
    a.vis_elems = (size_t)a.d.n_chan * (size_t)(n_in * (n_in + 1) / 2) * 2;
  }
  if (!s->dry) {
    if ((rc = cuda_err(cudaGetDevice(&s->device))) != CORR_OK ||
        (rc = cuda_err(cudaMalloc(&s->d_arena, arena_bytes))) != CORR_OK ||
        (rc = cuda_err(cudaStreamCreateWithFlags(&s->s_copy, cudaStreamNonBlocking))) !=
            CORR_OK ||
        (rc = cuda_err(cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking))) != CORR_OK) {
      free_server(s);
      return rc;
    }
    // CORR_SERVER_ONE_STREAM=1 puts every array's work on one compute stream
    // (a device queue in arrival order), for comparison
    const char *one = std::getenv("CORR_SERVER_ONE_STREAM");
    const bool shared = one && one[0] == '1';
    for (Array &a : s->arrays) {
      if (shared && &a != &s->arrays[0]) {
        a.s_compute = s->arrays[0].s_compute;
        a.stream_shared = true;
      } else if ((rc = cuda_err(cudaStreamCreateWithFlags(&a.s_compute, cudaStreamNonBlocking))) !=
                 CORR_OK) {
        free_server(s);
        return rc;
      }
      if ((rc = corr_create(a.d.n_ant, a.d.n_pol, a.d.n_chan, a.d.block_len, &a.ctx)) !=
              CORR_OK ||
          (rc = cuda_err(cudaMalloc(&a.d_vis, a.vis_elems * sizeof(int64_t)))) != CORR_OK ||
          (rc = cuda_err(cudaMallocHost(&a.h_vis, a.vis_elems * sizeof(int64_t)))) != CORR_OK ||
          (rc = cuda_err(cudaEventCreateWithFlags(&a.dumped, cudaEventDisableTiming))) !=
              CORR_OK) {
        free_server(s);
        return rc;
      }
    }
  }
  s->worker = std::thread([s] { s->run(); });
  *out = s;
  return CORR_OK;
}

int corr_server_submit(corr_server *s, int array, long long seq, const uint8_t *h_block) {
  if (!s || array < 0 || array >= (int)s->arrays.size() || seq < 0 || (!h_block && !s->dry))
    return CORR_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->error != CORR_OK) return s->error;
    s->inbox.push_back({array, seq, h_block, now_ms()});
    ++s->n_submitted;
  }
  s->cv_work.notify_one();
  return CORR_OK;
}

int corr_server_poll(corr_server *s, corr_result *out, int max_results, int timeout_ms) {
  if (!s || (!out && max_results > 0) || max_results < 0) return CORR_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  if (s->results.empty() && timeout_ms > 0)
    s->cv_results.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                           [s] { return !s->results.empty() || s->error != CORR_OK; });
  if (s->error != CORR_OK && s->results.empty()) return s->error;
  int n = 0;
  while (n < max_results && !s->results.empty()) {
    out[n++] = s->results.front();
    s->results.pop_front();
  }
  return n;
}

int corr_server_release(corr_server *s, int array) {
  if (!s || array < 0 || array >= (int)s->arrays.size()) return CORR_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->arrays[array].result_held = false;
  }
  s->cv_work.notify_one();
  return CORR_OK;
}

int corr_server_flush(corr_server *s) {
  if (!s) return CORR_EINVAL;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->flush_req = true;
  }
  s->cv_work.notify_one();
  return CORR_OK;
}

int corr_server_stats(corr_server *s, corr_server_info *out) {
  if (!s || !out) return CORR_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->n_submitted;
  out->integrated = s->n_integrated;
  out->duplicates = s->n_dup;
  out->late = s->n_late;
  out->integrations = s->n_integrations;
  out->incomplete_integrations = s->n_incomplete;
  out->latency_p50_ms = percentile(s->latencies, 0.50);
  out->latency_p99_ms = percentile(s->latencies, 0.99);
  out->latency_max_ms = s->latencies.empty()
                            ? 0.0
                            : *std::max_element(s->latencies.begin(), s->latencies.end());
  out->latency_samples = (long long)s->latencies.size();
  out->arena_peak_bytes = s->arena->peak();
  out->error = s->error;
  return CORR_OK;
}

void corr_server_destroy(corr_server *s) { free_server(s); }

}  // extern "C"
