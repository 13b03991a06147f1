// Batching and serving around the per-system calls.
//
// kkt_batch_factor_solve: independent arrowhead systems (each with its own
// analysed handle) are spread over a pool of CUDA streams, one host worker per
// stream; the refinement of each solve synchronizes only its own stream, so the
// kernels of different systems overlap on the GPU.
//
// kkt_server_*: a request loop with continuous batching.  Requests (a handle
// plus the values and right-hand side of one KKT solve) are queued on submit;
// up to `slots` requests are in flight, each on its own worker stream, and a new
// request is admitted as soon as a slot is free and its handle is not busy.
// Handles stay resident across requests (repeated solves of a pattern reuse
// its analysis and buffers).  Admission also checks that the handles in flight
// fit the device-memory budget given at creation.  Each request's latency runs
// from its submit to the completion of its solve.
//
// With a pattern cache (kkt_server_set_cache) a request may name a pattern
// instead of a handle: the server analyses it at its first request, keeps the
// handle resident for later requests on the same key (re-solves with new
// values) and admits new patterns by free device memory, evicting idle
// handles least recently used first.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "handle.h"

using namespace kkt;

extern "C" kkt_status kkt_batch_factor_solve(kkt_handle* const* handles, int32_t n,
                                             const double* const* a_vals, const double* const* b_vals,
                                             const double* const* c_vals, const double* const* rhs,
                                             double* const* x, int32_t on_device, int32_t streams,
                                             kkt_status* statuses) {
  if (n < 0 || (n > 0 && (!handles || !a_vals || !b_vals || !c_vals || !rhs || !x))) {
    set_error("kkt_batch_factor_solve: invalid argument");
    return KKT_ERR_INVALID;
  }
  if (n == 0) return KKT_OK;
  const int ns = std::max(1, std::min<int>(streams > 0 ? streams : 8, n));
  std::vector<cudaStream_t> pool(ns, nullptr);
  for (int s = 0; s < ns; s++) {
    cudaError_t e = cudaStreamCreateWithFlags(&pool[s], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int q = 0; q < s; q++) cudaStreamDestroy(pool[q]);
      set_error(std::string("kkt_batch_factor_solve: cudaStreamCreate: ") + cudaGetErrorString(e));
      return KKT_ERR_CUDA;
    }
  }
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<kkt_status> st(n, KKT_OK);
  std::vector<std::thread> workers;
  for (int s = 0; s < ns; s++) {
    workers.emplace_back([&, s]() {
      cudaSetDevice(dev);
      for (int i = s; i < n; i += ns) {  // round robin: system i on stream i mod ns
        kkt_status r = kkt_factor(handles[i], a_vals[i], b_vals[i], c_vals[i], on_device, pool[s]);
        if (r == KKT_OK) r = kkt_solve(handles[i], rhs[i], x[i], 1, on_device, pool[s]);
        st[i] = r;
      }
    });
  }
  for (auto& w : workers) w.join();
  for (int s = 0; s < ns; s++) cudaStreamDestroy(pool[s]);
  kkt_status worst = KKT_OK;
  for (int i = 0; i < n; i++) {
    if (statuses) statuses[i] = st[i];
    if (st[i] != KKT_OK && (worst == KKT_OK || worst == KKT_ERR_NOT_CONVERGED)) worst = st[i];
  }
  return worst;
}

namespace {

struct Request {
  int64_t id;
  kkt_handle* h;
  const double *a, *b, *c, *rhs;
  double* x;
  int32_t on_device;
  std::chrono::steady_clock::time_point t_submit;
  int64_t key = -1;                  // a cached pattern (h is null until the worker has its handle)
  const kkt_pattern* pat = nullptr;
};

// A pattern the server analysed at its first request and keeps resident.
struct CacheEntry {
  kkt_handle* h = nullptr;  // null while a worker analyses it
  bool busy = false;        // a request on it is running (or it is being analysed)
  uint64_t last_use = 0;    // for least-recently-used eviction
};

struct Done {
  kkt_status status;
  double latency_ms;
};

}  // namespace

struct kkt_server {
  int slots = 1;
  int64_t budget = 0;  // device bytes of handles that may be in flight at once (0 = no limit)
  int dev = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request> queue;
  std::unordered_map<int64_t, Done> done;
  std::unordered_set<kkt_handle*> busy;
  std::unordered_set<int64_t> running;  // ids taken by a worker, not yet done
  int64_t inflight_bytes = 0;
  int64_t next_id = 1;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  // pattern cache (kkt_server_set_cache / kkt_server_submit_pattern)
  bool cache_on = false;
  kkt_options cache_opt{};
  int64_t reserve_bytes = 0;
  std::unordered_map<int64_t, CacheEntry> cache;
  uint64_t use_clock = 0;
  int64_t analyses = 0, evictions = 0;
  std::mutex analyze_mu;  // one analysis (and its evictions) at a time
};

namespace {

// The handle of a cached pattern, analysed now if the server has none yet.
// Admission by free device memory: before the analysis, idle resident
// handles are evicted (least recently used first) while the free memory
// (cudaMemGetInfo) is below the reserve; an analysis that still runs out of
// memory evicts one more idle handle and retries, until none is left.
kkt_status obtain_cached(kkt_server* S, Request& req) {
  std::lock_guard<std::mutex> alk(S->analyze_mu);
  auto evict_one = [&]() -> bool {
    kkt_handle* victim = nullptr;
    int64_t vkey = 0;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      uint64_t best = UINT64_MAX;
      for (auto& kv : S->cache)
        if (!kv.second.busy && kv.second.h && kv.second.last_use < best) {
          best = kv.second.last_use;
          vkey = kv.first;
          victim = kv.second.h;
        }
      if (victim) {
        S->cache.erase(vkey);
        S->evictions++;
      }
    }
    if (victim) kkt_destroy(victim);
    return victim != nullptr;
  };
  for (;;) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) break;
    if ((int64_t)free_b >= S->reserve_bytes || !evict_one()) break;
  }
  kkt_handle* h = nullptr;
  kkt_status r;
  for (;;) {
    r = kkt_analyze(req.pat, &S->cache_opt, &h);
    if (r != KKT_ERR_OOM || !evict_one()) break;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (r == KKT_OK) {
    S->cache[req.key].h = h;
    S->analyses++;
  } else {
    S->cache.erase(req.key);  // a later request on the key tries again
  }
  req.h = h;
  return r;
}

void worker_loop(kkt_server* S, int slot) {
  cudaSetDevice(S->dev);
  for (;;) {
    Request req;
    int64_t bytes = 0;
    bool analyse = false;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->stop && S->queue.empty()) return;
        // the oldest queued request whose handle (or cached pattern) is idle and
        // which fits the budget
        auto it = S->queue.begin();
        for (; it != S->queue.end(); ++it) {
          if (it->key >= 0) {
            auto c = S->cache.find(it->key);
            if (c != S->cache.end() && c->second.busy) continue;
            break;
          }
          if (S->busy.count(it->h)) continue;
          const int64_t hb = reinterpret_cast<Handle*>(it->h)->device_bytes;
          if (S->budget > 0 && S->inflight_bytes > 0 && S->inflight_bytes + hb > S->budget) continue;
          break;
        }
        if (it != S->queue.end()) {
          req = *it;
          S->queue.erase(it);
          S->running.insert(req.id);
          if (req.key >= 0) {
            CacheEntry& c = S->cache[req.key];  // created (handle null) at its first request
            c.busy = true;
            c.last_use = ++S->use_clock;
            req.h = c.h;
            analyse = c.h == nullptr;
          } else {
            bytes = reinterpret_cast<Handle*>(req.h)->device_bytes;
            S->busy.insert(req.h);
            S->inflight_bytes += bytes;
          }
          break;
        }
        S->cv_work.wait(lk);
      }
    }
    cudaStream_t st = S->streams[slot];
    kkt_status r = analyse ? obtain_cached(S, req) : KKT_OK;
    if (r == KKT_OK) r = kkt_factor(req.h, req.a, req.b, req.c, req.on_device, st);
    if (r == KKT_OK) r = kkt_solve(req.h, req.rhs, req.x, 1, req.on_device, st);
    if (r == KKT_OK || r == KKT_ERR_NOT_CONVERGED) cudaStreamSynchronize(st);
    const double ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - req.t_submit).count();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      if (req.key >= 0) {
        auto c = S->cache.find(req.key);
        if (c != S->cache.end()) c->second.busy = false;
      } else {
        S->busy.erase(req.h);
        S->inflight_bytes -= bytes;
      }
      S->running.erase(req.id);
      S->done[req.id] = Done{r, ms};
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

}  // namespace

extern "C" kkt_status kkt_server_create(int32_t slots, int64_t device_budget_bytes, kkt_server** out) {
  if (!out || slots < 1) {
    set_error("kkt_server_create: invalid argument");
    return KKT_ERR_INVALID;
  }
  kkt_server* S = new (std::nothrow) kkt_server();
  if (!S) return KKT_ERR_OOM;
  S->slots = slots;
  S->budget = device_budget_bytes;
  cudaGetDevice(&S->dev);
  S->streams.resize(slots, nullptr);
  for (int s = 0; s < slots; s++) {
    cudaError_t e = cudaStreamCreateWithFlags(&S->streams[s], cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (int q = 0; q < s; q++) cudaStreamDestroy(S->streams[q]);
      delete S;
      set_error(std::string("kkt_server_create: cudaStreamCreate: ") + cudaGetErrorString(e));
      return KKT_ERR_CUDA;
    }
  }
  for (int s = 0; s < slots; s++) S->workers.emplace_back(worker_loop, S, s);
  *out = S;
  return KKT_OK;
}

extern "C" kkt_status kkt_server_submit(kkt_server* S, kkt_handle* h, const double* a_vals,
                                        const double* b_vals, const double* c_vals, const double* rhs,
                                        double* x, int32_t on_device, int64_t* request_id) {
  if (!S || !h || !a_vals || !rhs || !x || !request_id) {
    set_error("kkt_server_submit: invalid argument");
    return KKT_ERR_INVALID;
  }
  Request r{0, h, a_vals, b_vals, c_vals, rhs, x, on_device, std::chrono::steady_clock::now()};
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->stop) {
      set_error("kkt_server_submit: server is shutting down");
      return KKT_ERR_STATE;
    }
    r.id = S->next_id++;
    S->queue.push_back(r);
  }
  *request_id = r.id;
  S->cv_work.notify_one();
  return KKT_OK;
}

extern "C" kkt_status kkt_server_set_cache(kkt_server* S, const kkt_options* opt, int64_t reserve_bytes) {
  if (!S || reserve_bytes < 0) {
    set_error("kkt_server_set_cache: invalid argument");
    return KKT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  if (!S->cache.empty()) {
    set_error("kkt_server_set_cache: the cache already holds patterns");
    return KKT_ERR_STATE;
  }
  kkt_default_options(&S->cache_opt);
  if (opt) S->cache_opt = *opt;
  S->reserve_bytes = reserve_bytes;
  S->cache_on = true;
  return KKT_OK;
}

extern "C" kkt_status kkt_server_submit_pattern(kkt_server* S, int64_t key, const kkt_pattern* pat,
                                                const double* a_vals, const double* b_vals, const double* c_vals,
                                                const double* rhs, double* x, int32_t on_device,
                                                int64_t* request_id) {
  if (!S || key < 0 || !pat || !a_vals || !rhs || !x || !request_id) {
    set_error("kkt_server_submit_pattern: invalid argument");
    return KKT_ERR_INVALID;
  }
  Request r{0, nullptr, a_vals, b_vals, c_vals, rhs, x, on_device, std::chrono::steady_clock::now()};
  r.key = key;
  r.pat = pat;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->cache_on) {
      set_error("kkt_server_submit_pattern: no pattern cache (kkt_server_set_cache first)");
      return KKT_ERR_STATE;
    }
    if (S->stop) {
      set_error("kkt_server_submit_pattern: server is shutting down");
      return KKT_ERR_STATE;
    }
    r.id = S->next_id++;
    S->queue.push_back(r);
  }
  *request_id = r.id;
  S->cv_work.notify_one();
  return KKT_OK;
}

extern "C" kkt_status kkt_server_cache_info(kkt_server* S, int64_t* resident, int64_t* analyses,
                                            int64_t* evictions) {
  if (!S) {
    set_error("kkt_server_cache_info: null server");
    return KKT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  int64_t n = 0;
  for (auto& kv : S->cache) n += kv.second.h != nullptr;
  if (resident) *resident = n;
  if (analyses) *analyses = S->analyses;
  if (evictions) *evictions = S->evictions;
  return KKT_OK;
}

extern "C" kkt_status kkt_server_poll(kkt_server* S, int64_t request_id, int32_t wait, kkt_status* status,
                                      double* latency_ms) {
  if (!S) {
    set_error("kkt_server_poll: null server");
    return KKT_ERR_INVALID;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    auto it = S->done.find(request_id);
    if (it != S->done.end()) {
      if (status) *status = it->second.status;
      if (latency_ms) *latency_ms = it->second.latency_ms;
      S->done.erase(it);
      return KKT_OK;
    }
    // not finished: it must be queued or running
    bool pending = S->running.count(request_id) > 0;
    for (auto q = S->queue.begin(); !pending && q != S->queue.end(); ++q) pending = q->id == request_id;
    if (!pending) {
      set_error("kkt_server_poll: unknown or already collected request");
      return KKT_ERR_INVALID;
    }
    if (!wait) return KKT_ERR_STATE;
    S->cv_done.wait(lk);
  }
}

extern "C" kkt_status kkt_server_destroy(kkt_server* S) {
  if (!S) return KKT_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (auto& w : S->workers) w.join();
  for (cudaStream_t st : S->streams) cudaStreamDestroy(st);
  for (auto& kv : S->cache)
    if (kv.second.h) kkt_destroy(kv.second.h);
  delete S;
  return KKT_OK;
}
