// server.cu -- a request loop over the batched sieve with continuous batching.
//
// Clients submit [lo, hi) range queries from any thread; a server thread
// forms batches from the admitted requests and runs each as one batched
// launch (batch.cu) on one of two streams.  While one batch is on the GPU the
// next is formed from the requests that arrived meanwhile and launched on the
// other stream, so the tail of one batch overlaps the head of the next, and a
// request never waits for more than the batch in front of it.
//
// Admission is by device memory: a list-mode request reserves room for the
// largest possible answer in a device pool of fixed size when it is
// submitted, and gives it back when its result is collected; when the pool
// (or the queue) is full, submit returns SIEVE_ERR_BUSY (backpressure).  The
// base-prime table and the batch buffers stay on the device for the server's
// lifetime.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch.cuh"

namespace sieve {
namespace {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, n) elements of the device pool.
class PoolAllocator {
 public:
  explicit PoolAllocator(uint64_t n) {
    if (n) free_[0] = n;
  }
  bool alloc(uint64_t n, uint64_t *off) {
    *off = 0;
    if (n == 0) return true;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const uint64_t rest = it->second - n, o2 = it->first + n;
      free_.erase(it);
      if (rest) free_[o2] = rest;
      used_ += n;
      return true;
    }
    return false;
  }
  void release(uint64_t off, uint64_t n) {
    if (n == 0) return;
    used_ -= n;
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  uint64_t used() const { return used_; }

 private:
  std::map<uint64_t, uint64_t> free_;
  uint64_t used_ = 0;
};

enum ReqState : int { kQueued = 0, kInFlight = 1, kDone = 2 };

struct Request {
  uint64_t lo = 0, hi = 0;
  uint8_t mode = 0;
  int state = kQueued;
  int status = SIEVE_OK;
  uint64_t res_off = 0, res_len = 0;  // list reservation in the pool (elements)
  sieve_count_result cnt{0, 0};
  uint64_t n = 0;
  Clock::time_point t_submit, t_done;
};

// Upper bound on the number of primes in a range of width w, for the list
// reservation: among w consecutive integers at most 2 ceil(w / 6) are prime
// to 6, plus 2 and 3; and pi(x + w) - pi(x) <= 2 w / ln w for w > 1
// (Montgomery & Vaughan, "The large sieve", 1973), used here with slack.  The
// kernels check every query's count against its reservation as well.
uint64_t list_bound(uint64_t w) {
  if (w == 0) return 0;
  const uint64_t a = 2 * ((w + 5) / 6) + 2;
  if (w < 64) return a;
  const double b = 2.0 * (double)w / std::log((double)w) + 64.0;
  return std::min<uint64_t>(a, (uint64_t)b);
}

// Scratch a request adds to a batch (bytes): its tiles' bitmaps, for list
// output and for merged tiles, about one bit per candidate each.
uint64_t scratch_estimate(uint64_t w) { return w / 12 + 4096; }

}  // namespace
}  // namespace sieve

using namespace sieve;

struct sieve_server {
  sieve_ctx *ctx = nullptr;
  sieve_server_config cfg{};
  uint64_t *d_pool = nullptr;
  uint64_t pool_elems = 0;
  PoolAllocator *pool = nullptr;
  struct Slot {
    BatchRunner *runner = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> ids;
    std::vector<uint64_t> lo, hi, base, cap;
    std::vector<uint8_t> mode;
    sieve_count_result *h_cnt = nullptr;  // pinned, max_batch
    uint64_t *h_off = nullptr;            // pinned, max_batch + 1
    BatchState *h_state = nullptr;        // pinned
    uint32_t *h_yield = nullptr;          // pinned: id of this slot's batch, for a yield request
  } slots[2];
  cudaStream_t collect = nullptr;
  std::mutex mu;
  std::condition_variable cv;       // loop: new work or stop
  std::condition_variable done_cv;  // clients: completions
  std::deque<uint64_t> queue;
  std::unordered_map<uint64_t, Request> reqs;
  std::deque<uint64_t> done_ids;
  uint64_t next_id = 1;
  bool stop = false;
  int fatal = SIEVE_OK;
  std::string fatal_msg;
  std::thread th;
  uint64_t completed = 0, rejected = 0, batches = 0, batched = 0, overlapped = 0;
  std::vector<double> lat_us;
};

namespace {

void fail_requests(sieve_server *s, const std::vector<uint64_t> &ids, int status) {
  const auto now = Clock::now();
  for (uint64_t id : ids) {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) continue;
    it->second.state = kDone;
    it->second.status = status;
    it->second.t_done = now;
    s->done_ids.push_back(id);
  }
  s->done_cv.notify_all();
}

// Results of a finished batch (lock held).
void finish_slot(sieve_server *s, sieve_server::Slot &sl) {
  const auto now = Clock::now();
  for (size_t i = 0; i < sl.ids.size(); i++) {
    auto it = s->reqs.find(sl.ids[i]);
    if (it == s->reqs.end()) continue;
    Request &r = it->second;
    r.cnt = sl.h_cnt[i];
    r.n = sl.h_off[i + 1] - sl.h_off[i];
    if (r.mode == SIEVE_LIST && r.n > r.res_len) r.status = SIEVE_ERR_CAPACITY;  // not written (kernel check)
    r.state = kDone;
    r.t_done = now;
    s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t_submit).count());
    s->done_ids.push_back(sl.ids[i]);
    s->completed++;
  }
  sl.ids.clear();
  sl.busy = false;
  s->done_cv.notify_all();
}

// Form a batch from the queue and launch it on slot sl (called with the lock
// held; drops it while planning and launching).
void launch_slot(sieve_server *s, sieve_server::Slot &sl, std::unique_lock<std::mutex> &lk) {
  sl.ids.clear();
  sl.lo.clear();
  sl.hi.clear();
  sl.mode.clear();
  sl.base.clear();
  sl.cap.clear();
  uint64_t scratch = 0;
  while (!s->queue.empty() && sl.ids.size() < s->cfg.max_batch) {
    const uint64_t id = s->queue.front();
    Request &r = s->reqs[id];
    const uint64_t sc = scratch_estimate(r.hi - r.lo);
    if (!sl.ids.empty() && scratch + sc > s->cfg.batch_scratch_bytes) break;
    s->queue.pop_front();
    scratch += sc;
    r.state = kInFlight;
    sl.ids.push_back(id);
    sl.lo.push_back(r.lo);
    sl.hi.push_back(r.hi);
    sl.mode.push_back(r.mode);
    sl.base.push_back(r.res_off);
    sl.cap.push_back(r.res_len);
  }
  if (sl.ids.empty()) return;
  sieve_server::Slot &other = &sl == &s->slots[0] ? s->slots[1] : s->slots[0];
  const bool other_busy = other.busy;
  sl.busy = true;
  lk.unlock();
  BatchRunner &rn = *sl.runner;
  const size_t n = sl.ids.size();
  int rc = batch_configure(rn);
  if (rc == SIEVE_OK)
    rc = batch_plan(rn, sl.lo.data(), sl.hi.data(), sl.mode.data(), n, s->d_pool, 0, 1, sl.base.data(),
                    sl.cap.data());
  if (rc == SIEVE_OK) rc = batch_prepare(rn);
  if (rc == SIEVE_OK) rc = batch_launch(rn);
  cudaError_t e = cudaSuccess;
  if (rc == SIEVE_OK &&
      ((e = cudaMemcpyAsync(sl.h_cnt, rn.d_acc, n * sizeof(sieve_count_result), cudaMemcpyDeviceToHost,
                            sl.stream)) != cudaSuccess ||
       (e = cudaMemcpyAsync(sl.h_off, rn.d_offsets, (n + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                            sl.stream)) != cudaSuccess ||
       (e = cudaMemcpyAsync(sl.h_state, rn.d_state, sizeof(BatchState), cudaMemcpyDeviceToHost, sl.stream)) !=
           cudaSuccess ||
       (e = cudaEventRecord(sl.done, sl.stream)) != cudaSuccess))
    rc = cuda_fail(e, "server batch read-back");
  const std::string msg = rc == SIEVE_OK ? std::string() : std::string(sieve_last_error());
  lk.lock();
  if (rc != SIEVE_OK) {
    sl.busy = false;
    fail_requests(s, sl.ids, rc);
    sl.ids.clear();
    if (rc == SIEVE_ERR_CUDA) {
      s->fatal = rc;
      s->fatal_msg = msg;
    }
    return;
  }
  s->batches++;
  s->batched += n;
  if (other_busy) {
    // the batch on the other stream may hold every SM: ask the upper half of
    // its CTAs to stop taking items, so that this batch starts now (best
    // effort: the copy may land after that batch ended, which is harmless)
    s->overlapped++;
    *other.h_yield = other.runner->batch_id;
    cudaMemcpyAsync(&other.runner->d_state->yield_batch, other.h_yield, sizeof(uint32_t), cudaMemcpyHostToDevice,
                    s->collect);
  }
}

void server_loop(sieve_server *s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    bool progressed = false;
    bool any_busy = false;
    for (auto &sl : s->slots) {
      if (!sl.busy || sl.ids.empty()) continue;
      const cudaError_t q = cudaEventQuery(sl.done);
      if (q == cudaSuccess) {
        finish_slot(s, sl);
        progressed = true;
      } else if (q != cudaErrorNotReady) {
        s->fatal = cuda_fail(q, "server batch");
        s->fatal_msg = sieve_last_error();
        sl.busy = false;
        fail_requests(s, sl.ids, SIEVE_ERR_CUDA);
        sl.ids.clear();
      } else {
        any_busy = true;
      }
    }
    if (s->stop && s->queue.empty() && !any_busy) break;
    if (s->fatal == SIEVE_OK) {
      for (auto &sl : s->slots) {
        if (!sl.busy && !s->queue.empty()) {
          launch_slot(s, sl, lk);
          progressed = true;
          any_busy = any_busy || sl.busy;
        }
      }
    } else if (!s->queue.empty()) {
      std::vector<uint64_t> ids(s->queue.begin(), s->queue.end());
      s->queue.clear();
      fail_requests(s, ids, s->fatal);
    }
    if (progressed) continue;
    if (any_busy) {
      // a batch is on the GPU: look again shortly, or at once on a submit
      s->cv.wait_for(lk, std::chrono::microseconds(20));
    } else {
      s->cv.wait(lk, [&] { return s->stop || !s->queue.empty(); });
    }
  }
}

void free_server(sieve_server *s) {
  for (auto &sl : s->slots) {
    destroy_batch_runner(sl.runner);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.h_cnt) cudaFreeHost(sl.h_cnt);
    if (sl.h_off) cudaFreeHost(sl.h_off);
    if (sl.h_state) cudaFreeHost(sl.h_state);
    if (sl.h_yield) cudaFreeHost(sl.h_yield);
  }
  if (s->collect) cudaStreamDestroy(s->collect);
  cudaFree(s->d_pool);
  delete s->pool;
  delete s;
}

}  // namespace

extern "C" int sieve_server_start(sieve_ctx *ctx, const sieve_server_config *config, sieve_server **srv) {
  if (!ctx || !srv) {
    set_error("sieve_server_start: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  *srv = nullptr;
  sieve_server_config cfg{};
  if (config) cfg = *config;
  if (cfg.max_batch == 0) cfg.max_batch = 4096;
  if (cfg.max_queue == 0) cfg.max_queue = 1u << 16;
  if (cfg.batch_scratch_bytes == 0) cfg.batch_scratch_bytes = 1ull << 30;
  if (cfg.max_batch > (1u << 20)) {
    set_error("max_batch must be <= 2^20");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  sieve_server *s = new (std::nothrow) sieve_server();
  if (!s) {
    set_error("host allocation failed");
    return SIEVE_ERR_OOM;
  }
  s->ctx = ctx;
  s->cfg = cfg;
  int rc = SIEVE_OK;
  do {
    cudaError_t e;
    s->pool_elems = cfg.pool_bytes / sizeof(uint64_t);
    if (s->pool_elems && (e = cudaMalloc(&s->d_pool, s->pool_elems * sizeof(uint64_t))) != cudaSuccess) {
      rc = cuda_fail(e, "server pool");
      break;
    }
    s->pool = new (std::nothrow) PoolAllocator(s->pool_elems);
    if (!s->pool || (e = cudaStreamCreateWithFlags(&s->collect, cudaStreamNonBlocking)) != cudaSuccess) {
      rc = s->pool ? cuda_fail(e, "server stream") : SIEVE_ERR_OOM;
      break;
    }
    for (auto &sl : s->slots) {
      if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaMallocHost((void **)&sl.h_cnt, cfg.max_batch * sizeof(sieve_count_result))) != cudaSuccess ||
          (e = cudaMallocHost((void **)&sl.h_off, (cfg.max_batch + 1) * sizeof(uint64_t))) != cudaSuccess ||
          (e = cudaMallocHost((void **)&sl.h_state, sizeof(BatchState))) != cudaSuccess ||
          (e = cudaMallocHost((void **)&sl.h_yield, sizeof(uint32_t))) != cudaSuccess) {
        rc = cuda_fail(e, "server slot");
        break;
      }
      sl.runner = new_batch_runner(ctx, sl.stream);
      if (!sl.runner) {
        rc = SIEVE_ERR_OOM;
        break;
      }
      if ((rc = batch_configure(*sl.runner)) != SIEVE_OK) break;
      // buffers for a full batch now: growing one later would free the old
      // buffer, and cudaFree waits for the batch running on the other stream
      if ((rc = batch_reserve(*sl.runner, cfg.max_batch, 16 * cfg.max_batch + 65536,
                              cfg.batch_scratch_bytes / 2 / sizeof(uint32_t),
                              cfg.batch_scratch_bytes / 2 / sizeof(uint2))) != SIEVE_OK)
        break;
    }
    if (rc != SIEVE_OK) break;
    // every tile width's presieve patterns now, so that the loop never builds
    // them on the context's stream
    for (uint32_t lw = 5; lw + 5 <= s->slots[0].runner->logLmax; lw++)
      if ((rc = ensure_pattern_set_dev(ctx, lw)) != SIEVE_OK) break;
  } while (0);
  if (rc != SIEVE_OK) {
    free_server(s);
    return rc;
  }
  s->th = std::thread(server_loop, s);
  *srv = s;
  return SIEVE_OK;
}

extern "C" int sieve_server_submit(sieve_server *s, uint64_t lo, uint64_t hi, int mode, uint64_t *req_id) {
  if (!s || !req_id) {
    set_error("sieve_server_submit: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  if (lo > hi || (mode != SIEVE_COUNT && mode != SIEVE_LIST)) {
    set_error("sieve_server_submit: lo > hi or bad mode");
    return SIEVE_ERR_INVALID;
  }
  if (hi > (1ull << 63) || (hi > lo && isqrt_u64(hi - 1) > s->ctx->table.limit)) {
    set_error("sieve_server_submit: hi beyond the base table");
    return SIEVE_ERR_RANGE;
  }
  const uint64_t need = mode == SIEVE_LIST ? list_bound(hi - lo) : 0;
  if (need > s->pool_elems) {
    set_error("sieve_server_submit: a list of up to %llu primes exceeds the server's pool of %llu",
              (unsigned long long)need, (unsigned long long)s->pool_elems);
    return SIEVE_ERR_CAPACITY;
  }
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    set_error("server is stopping");
    return SIEVE_ERR_INVALID;
  }
  if (s->fatal != SIEVE_OK) {
    set_error("server failed: %s", s->fatal_msg.c_str());
    return s->fatal;
  }
  uint64_t off = 0;
  if (s->queue.size() >= s->cfg.max_queue || !s->pool->alloc(need, &off)) {
    s->rejected++;
    set_error("server busy: queue or device pool full");
    return SIEVE_ERR_BUSY;
  }
  const uint64_t id = s->next_id++;
  Request &r = s->reqs[id];
  r.lo = lo;
  r.hi = hi;
  r.mode = (uint8_t)mode;
  r.res_off = off;
  r.res_len = need;
  r.t_submit = Clock::now();
  s->queue.push_back(id);
  s->cv.notify_one();
  *req_id = id;
  return SIEVE_OK;
}

extern "C" int sieve_server_poll(sieve_server *s, uint64_t req_id, sieve_count_result *cnt, uint64_t *out,
                                 size_t cap, size_t *n_out, unsigned flags) {
  if (!s) {
    set_error("sieve_server_poll: NULL server");
    return SIEVE_ERR_INVALID;
  }
  uint64_t off = 0, len = 0, n = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) {
      set_error("request %llu unknown or already collected", (unsigned long long)req_id);
      return SIEVE_ERR_NOT_FOUND;
    }
    Request &r = it->second;
    if (r.state != kDone) return SIEVE_PENDING;
    if (cnt) *cnt = r.cnt;
    if (n_out) *n_out = (size_t)r.n;
    if (r.status != SIEVE_OK) {
      const int st = r.status;
      s->pool->release(r.res_off, r.res_len);
      s->reqs.erase(it);
      set_error("request %llu failed", (unsigned long long)req_id);
      return st;
    }
    if (r.mode == SIEVE_LIST && r.n > 0) {
      if (!out || cap < r.n) {
        set_error("output capacity %zu is below the %llu primes listed", cap, (unsigned long long)r.n);
        return SIEVE_ERR_CAPACITY;  // the request stays; poll again with a larger buffer
      }
    }
    off = r.res_off;
    len = r.res_len;
    n = r.mode == SIEVE_LIST ? r.n : 0;
    s->reqs.erase(it);
  }
  int rc = SIEVE_OK;
  if (n) {
    cudaError_t e = cudaSetDevice(s->ctx->device);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out, s->d_pool + off, n * sizeof(uint64_t),
                          (flags & SIEVE_OUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->collect);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->collect);
    if (e != cudaSuccess) rc = cuda_fail(e, "server collect");
  }
  std::lock_guard<std::mutex> lk(s->mu);
  s->pool->release(off, len);
  return rc;
}

extern "C" int sieve_server_next_done(sieve_server *s, uint64_t *req_id, int timeout_us) {
  if (!s || !req_id) {
    set_error("sieve_server_next_done: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done_ids.empty() && timeout_us > 0)
    s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->done_ids.empty(); });
  if (s->done_ids.empty()) return SIEVE_PENDING;
  *req_id = s->done_ids.front();
  s->done_ids.pop_front();
  return SIEVE_OK;
}

extern "C" int sieve_server_get_stats(sieve_server *s, sieve_server_stats *st, int reset) {
  if (!s || !st) {
    set_error("sieve_server_get_stats: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  std::vector<double> lat;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->batches = s->batches;
    st->overlapped_batches = s->overlapped;
    st->mean_batch = s->batches ? (double)s->batched / (double)s->batches : 0.0;
    st->pool_used_bytes = s->pool->used() * sizeof(uint64_t);
    st->queued = s->queue.size();
    lat = s->lat_us;
    if (reset) {
      s->completed = s->rejected = s->batches = s->batched = s->overlapped = 0;
      s->lat_us.clear();
    }
  }
  if (!lat.empty()) {
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double p) {
      const size_t k = (size_t)std::min<double>((double)lat.size() - 1, std::ceil(p * (double)lat.size()) - 1);
      return lat[k];
    };
    double sum = 0;
    for (double x : lat) sum += x;
    st->p50_us = pct(0.50);
    st->p99_us = pct(0.99);
    st->mean_us = sum / (double)lat.size();
    st->max_us = lat.back();
  }
  return SIEVE_OK;
}

extern "C" void sieve_server_stop(sieve_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->th.joinable()) s->th.join();
  cudaSetDevice(s->ctx->device);
  for (auto &sl : s->slots)
    if (sl.stream) cudaStreamSynchronize(sl.stream);
  free_server(s);
}
