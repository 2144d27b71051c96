// Serving form: a request loop that solves APSP requests of different sizes
// and element types as they arrive (continuous batching).
//
//   submit  copies the caller's matrix (host or device memory) into pinned
//           staging memory and queues the request (the caller keeps
//           ownership of its buffer);
//   the scheduler thread admits queued requests, oldest first, while an
//           in-flight slot is free and the request's device footprint fits the
//           HBM budget; each admitted request is uploaded once and solved on
//           its device-resident copy; requests with n <= 512 admitted together
//           (at least 8 of one element type) are solved by one batched
//           launch, the others by the multi-CTA path on a stream of their
//           own, so requests overlap on the device;
//           the result is copied back to pinned memory, the device buffer is
//           released in stream order, and a host callback marks completion
//           (latency = submit -> result in host memory);
//   poll / wait deliver the result into the caller's buffer (host or device
//           memory).
// A request's result is the same whether it is solved alone or in a mix:
// integer results are exact, and fp32 requests get the same per-element
// operations in the same stage order (s = 64 up to n = 512) from the batched
// and the multi-CTA kernels.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_internal.h"

struct apsp_server;

namespace apsp {
namespace {

using Clock = std::chrono::steady_clock;

int esize(int dtype) { return dtype == APSP_I16 ? 2 : 4; }
int64_t dev_ld(int64_t n, int dtype) {
  const int64_t q = 16 / esize(dtype);  // 16-byte rows: the TMA kernels apply
  return (n + q - 1) / q * q;
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Server;

struct Request {
  Server *srv = nullptr;
  uint64_t id = 0;
  int dtype = 0;
  int64_t n = 0, ld = 0;  // staging / device leading dimension
  size_t bytes = 0;       // n * ld * elem
  void *host = nullptr;   // pinned: the input, then the result
  size_t host_cap = 0;
  void *dev = nullptr;
  int64_t footprint = 0;
  std::atomic<int> state{kQueued};
  int status = APSP_OK;
  Clock::time_point t_submit, t_done;
};

struct Server {
  apsp_server_config cfg{};
  std::mutex mu;
  std::condition_variable cv;       // scheduler wake-ups
  std::condition_variable done_cv;  // waiters
  std::deque<Request *> queue;
  std::unordered_map<uint64_t, Request *> table;
  uint64_t next_id = 1;
  bool stop = false;
  int64_t bytes_resident = 0;
  int inflight = 0;
  std::vector<cudaStream_t> streams;  // [0]: batched launches; the rest: one large request each, round robin
  std::vector<void *> workspaces;     // per stream, for apsp_fw_ex
  int64_t ws_bytes = 0;
  size_t next_stream = 1;
  std::vector<double> lat_ms;
  int64_t submitted = 0, completed = 0, failed = 0;
  Clock::time_point t_first, t_last;
  bool any = false;
  std::multimap<size_t, void *> pinned_free;  // pinned buffers by size class
  void *desc_dev = nullptr;
  size_t desc_cap = 0;
  std::thread sched;
};

bool pinned_take(Server *s, size_t bytes, void **p, size_t *cap) {  // with s->mu held
  size_t c = 4096;
  while (c < bytes) c <<= 1;
  auto it = s->pinned_free.find(c);
  *cap = c;
  if (it == s->pinned_free.end()) return false;
  *p = it->second;
  s->pinned_free.erase(it);
  return true;
}

// Runs on a CUDA callback thread: no CUDA calls in here.
void CUDART_CB on_done(void *arg) {
  Request *r = static_cast<Request *>(arg);
  Server *s = r->srv;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = Clock::now();
    s->bytes_resident -= r->footprint;
    s->inflight -= 1;
    if (r->status == APSP_OK) {
      s->completed += 1;
      s->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
    } else {
      s->failed += 1;
    }
    s->t_last = r->t_done;
    r->state = r->status == APSP_OK ? kDone : kFailed;  // last: a waiter may free r from here on
  }
  s->cv.notify_all();
  s->done_cv.notify_all();
}

// Records a launch failure; the request completes (as failed) when its host
// callback runs, so that nobody frees it while the stream still refers to it.
void fail(Request *r, int rc) {
  if (r->status == APSP_OK) r->status = rc;
}

// Launches admitted requests (called without s->mu).
// Small requests of one element type below this count in one admission round
// are solved one by one on all SMs rather than one CTA each: the batched
// kernel pays off when it has many graphs to spread over the SMs.  The
// choice never changes a result: integer results are exact either way, and
// fp32 requests take the s = 64 batched shape, whose per-element operations
// and stage order are those of the single-graph path at s = 64.
constexpr int kMinBatch = 8;

void launch_admitted(Server *s, std::vector<Request *> &adm) {
  int small_count[3] = {0, 0, 0};
  auto dt_slot = [](int dtype) { return dtype == APSP_F32 ? 1 : dtype == APSP_I16 ? 2 : 0; };
  for (Request *r : adm)
    if (r->n <= kBatchCtaMaxN) ++small_count[dt_slot(r->dtype)];
  std::vector<Request *> small;
  for (Request *r : adm) {
    if (r->n <= kBatchCtaMaxN && small_count[dt_slot(r->dtype)] >= kMinBatch) {
      small.push_back(r);
      continue;
    }
    const size_t si = s->next_stream;
    s->next_stream = 1 + (s->next_stream % (s->streams.size() - 1));
    cudaStream_t st = s->streams[si];
    int rc = cudaMallocAsync(&r->dev, r->bytes, st) == cudaSuccess ? APSP_OK : APSP_ENOMEM;
    if (rc == APSP_OK && cudaMemcpyAsync(r->dev, r->host, r->bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      rc = APSP_ECUDA;
    if (rc == APSP_OK) {
      apsp_options o{};
      o.flags = APSP_FLAG_NO_GRAPH;  // device addresses change from request to request
      if (r->n <= kBatchCtaMaxN) o.kblock = 64;  // the batched kernels' depth: same result either way
      o.workspace = s->workspaces[si];
      o.workspace_bytes = s->ws_bytes;
      rc = apsp_fw_ex(r->dev, r->n, r->ld, r->dtype, &o, st);
    }
    if (rc == APSP_OK && cudaMemcpyAsync(r->host, r->dev, r->bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      rc = APSP_ECUDA;
    if (r->dev) cudaFreeAsync(r->dev, st);
    if (rc != APSP_OK) fail(r, rc);
    cudaLaunchHostFunc(st, on_done, r);
  }
  if (small.empty()) return;
  cudaStream_t st = s->streams[0];
  for (int dt : {APSP_I32, APSP_F32, APSP_I16}) {
    std::vector<Request *> grp;
    for (Request *r : small)
      if (r->dtype == dt) grp.push_back(r);
    if (grp.empty()) continue;
    std::stable_sort(grp.begin(), grp.end(), [](Request *a, Request *b) { return a->n > b->n; });
    int rc = APSP_OK;
    for (Request *r : grp) {
      if (rc == APSP_OK && cudaMallocAsync(&r->dev, r->bytes, st) != cudaSuccess) rc = APSP_ENOMEM;
      if (rc == APSP_OK && cudaMemcpyAsync(r->dev, r->host, r->bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = APSP_ECUDA;
    }
    if (rc == APSP_OK) {
      std::vector<BatchDesc> descs;
      for (Request *r : grp) descs.push_back({r->dev, r->ld, r->n});
      rc = run_batched_direct(descs.data(), (int)descs.size(), dt, st, &s->desc_dev, &s->desc_cap,
                              /*match_single=*/dt == APSP_F32);
    }
    for (Request *r : grp) {
      if (rc == APSP_OK && cudaMemcpyAsync(r->host, r->dev, r->bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = APSP_ECUDA;
      if (r->dev) cudaFreeAsync(r->dev, st);
      if (rc != APSP_OK) fail(r, rc);
      cudaLaunchHostFunc(st, on_done, r);
    }
  }
}

bool admissible(const Server *s, const Request *r) {
  if (s->inflight >= s->cfg.max_inflight) return false;
  return s->bytes_resident + r->footprint <= s->cfg.hbm_budget_bytes;
}

void scheduler(Server *s) {
  cudaSetDevice(s->cfg.device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv.wait(lk, [&] { return s->stop || (!s->queue.empty() && admissible(s, s->queue.front())); });
    if (s->stop) {
      for (Request *r : s->queue) {  // never admitted
        r->status = APSP_EBUSY;
        r->state = kFailed;
      }
      s->queue.clear();
      s->done_cv.notify_all();
      return;
    }
    std::vector<Request *> adm;
    while (!s->queue.empty() && admissible(s, s->queue.front())) {
      Request *r = s->queue.front();
      s->queue.pop_front();
      r->state = kRunning;
      s->inflight += 1;
      s->bytes_resident += r->footprint;
      adm.push_back(r);
    }
    lk.unlock();
    launch_admitted(s, adm);
    lk.lock();
  }
}

// Row-by-row copy between host matrices of different leading dimensions.
// Large matrices are split into row ranges copied by several host threads: a
// single core moves a 64 MiB matrix in several milliseconds, which would
// stall the submitting (or collecting) thread and every request behind it.
void copy_rows(void *dst, int64_t dld, const void *src, int64_t sld, int64_t n, int es) {
  auto range = [&](int64_t i0, int64_t i1) {
    for (int64_t i = i0; i < i1; ++i)
      memcpy(static_cast<char *>(dst) + i * dld * es, static_cast<const char *>(src) + i * sld * es,
             (size_t)n * es);
  };
  constexpr size_t kParallelBytes = 4u << 20;
  const size_t bytes = (size_t)n * n * es;
  const int hw = (int)std::thread::hardware_concurrency();
  const int parts = bytes < kParallelBytes ? 1 : std::max(1, std::min(8, hw / 2));
  if (parts <= 1) {
    range(0, n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t per = (n + parts - 1) / parts;
  for (int p = 1; p < parts; ++p) {
    const int64_t i0 = p * per, i1 = std::min<int64_t>(n, i0 + per);
    if (i0 < i1) th.emplace_back(range, i0, i1);
  }
  range(0, std::min<int64_t>(n, per));
  for (auto &t : th) t.join();
}

// Whether p is device memory of some GPU (not host, pinned or not).
bool on_device(const void *p) {
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();  // an unregistered host pointer on older runtimes
    return false;
  }
  return pa.type == cudaMemoryTypeDevice;
}

// Copies an n x n matrix between a caller's buffer and a pinned staging
// buffer; the caller's side may be host or device memory.
int copy_matrix(void *dst, int64_t dld, const void *src, int64_t sld, int64_t n, int es, bool device_side) {
  if (!device_side) {
    copy_rows(dst, dld, src, sld, n, es);
    return APSP_OK;
  }
  return cudaMemcpy2D(dst, (size_t)dld * es, src, (size_t)sld * es, (size_t)n * es, (size_t)n, cudaMemcpyDefault) ==
                 cudaSuccess
             ? APSP_OK
             : APSP_ECUDA;
}

// Delivers a finished request and frees it.  Called with the lock `lk` on
// s->mu held: the request leaves the table under the lock, its result is
// copied out with the lock released (a large copy must not hold up the
// scheduler or other waiters), and its staging buffer goes back to the pool
// under the lock again.  Returns with the lock released.
int deliver(Server *s, Request *r, void *out, int64_t out_ld, std::unique_lock<std::mutex> &lk) {
  int rc = r->state.load() == kDone ? APSP_OK : r->status;
  s->table.erase(r->id);
  lk.unlock();
  if (rc == APSP_OK && out && r->n > 0)
    rc = copy_matrix(out, out_ld, r->host, r->ld, r->n, esize(r->dtype), on_device(out));
  if (r->host) {
    std::lock_guard<std::mutex> g(s->mu);
    s->pinned_free.emplace(r->host_cap, r->host);
  }
  delete r;
  return rc;
}

}  // namespace
}  // namespace apsp

using namespace apsp;

struct apsp_server {
  Server s;
};

extern "C" int apsp_server_create(apsp_server **out, const apsp_server_config *cfg) {
  if (!out || !cfg || cfg->max_inflight <= 0 || cfg->hbm_budget_bytes <= 0 || cfg->streams < 0 || cfg->max_n <= 0)
    return APSP_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) return APSP_EINVAL;
  apsp_server *h = new apsp_server;
  Server *s = &h->s;
  s->cfg = *cfg;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(cfg->device);
  int rc = APSP_OK;
  const int nstreams = 1 + std::max(1, cfg->streams ? cfg->streams : 4);
  s->ws_bytes = std::max(apsp_workspace_bytes(cfg->max_n, APSP_F32, 0), apsp_workspace_bytes(cfg->max_n, APSP_I16, 0));
  for (int i = 0; i < nstreams && rc == APSP_OK; ++i) {
    cudaStream_t st = nullptr;
    void *ws = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) rc = APSP_ECUDA;
    if (rc == APSP_OK && s->ws_bytes && cudaMalloc(&ws, (size_t)s->ws_bytes) != cudaSuccess) rc = APSP_ENOMEM;
    s->streams.push_back(st);
    s->workspaces.push_back(ws);
  }
  // keep freed stream-ordered allocations in the pool between requests
  cudaMemPool_t pool;
  if (rc == APSP_OK && cudaDeviceGetDefaultMemPool(&pool, cfg->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaSetDevice(prev);
  if (rc != APSP_OK) {
    for (auto st : s->streams)
      if (st) cudaStreamDestroy(st);
    for (auto w : s->workspaces)
      if (w) cudaFree(w);
    delete h;
    return rc;
  }
  s->sched = std::thread(scheduler, s);
  *out = h;
  return APSP_OK;
}

extern "C" int apsp_submit(apsp_server *h, const void *host_dist, int64_t n, int64_t ld, int dtype, int flags,
                           uint64_t *ticket) {
  if (!h || !ticket || n < 0 || ld < n || (n > 0 && !host_dist) || flags != 0) return APSP_EINVAL;
  if (dtype != APSP_I32 && dtype != APSP_F32 && dtype != APSP_I16) return APSP_EINVAL;
  Server *s = &h->s;
  if (n > s->cfg.max_n) return APSP_EUNSUPPORTED;
  Request *r = new Request;
  r->srv = s;
  r->dtype = dtype;
  r->n = n;
  r->ld = dev_ld(std::max<int64_t>(n, 1), dtype);
  r->bytes = (size_t)n * r->ld * esize(dtype);
  r->footprint = (int64_t)r->bytes;
  if (r->footprint > s->cfg.hbm_budget_bytes) {
    delete r;
    return APSP_ENOMEM;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    pinned_take(s, std::max<size_t>(r->bytes, 1), &r->host, &r->host_cap);
  }
  if (!r->host && cudaMallocHost(&r->host, r->host_cap) != cudaSuccess) {
    delete r;
    return APSP_ENOMEM;
  }
  if (n > 0 && copy_matrix(r->host, r->ld, host_dist, ld, n, esize(dtype), on_device(host_dist)) != APSP_OK) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->pinned_free.emplace(r->host_cap, r->host);
    delete r;
    return APSP_ECUDA;
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
      s->pinned_free.emplace(r->host_cap, r->host);
      delete r;
      return APSP_EBUSY;
    }
    r->id = s->next_id++;
    r->t_submit = Clock::now();
    if (!s->any) {
      s->any = true;
      s->t_first = r->t_submit;
    }
    s->submitted += 1;
    s->table[r->id] = r;
    *ticket = r->id;
    if (n == 0) {  // nothing to solve
      r->state = kDone;
      r->t_done = r->t_submit;
      s->completed += 1;
      s->lat_ms.push_back(0.0);
    } else {
      s->queue.push_back(r);
    }
  }
  s->cv.notify_all();
  return APSP_OK;
}

extern "C" int apsp_poll(apsp_server *h, uint64_t ticket, void *out_dist, int64_t out_ld) {
  if (!h) return APSP_EINVAL;
  Server *s = &h->s;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return APSP_EINVAL;
  Request *r = it->second;
  const int st = r->state.load();
  if (st == kQueued || st == kRunning) return APSP_EPENDING;
  if (st == kDone && out_dist && out_ld < r->n) return APSP_EINVAL;
  return deliver(s, r, out_dist, out_ld, lk);
}

extern "C" int apsp_wait(apsp_server *h, uint64_t ticket, void *out_dist, int64_t out_ld, int64_t timeout_us) {
  if (!h) return APSP_EINVAL;
  Server *s = &h->s;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->table.find(ticket);
  if (it == s->table.end()) return APSP_EINVAL;
  Request *r = it->second;
  auto finished = [&] { return r->state.load() >= kDone; };
  if (timeout_us < 0)
    s->done_cv.wait(lk, finished);
  else if (!s->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), finished))
    return APSP_ETIMEOUT;
  if (r->state.load() == kDone && out_dist && out_ld < r->n) return APSP_EINVAL;
  return deliver(s, r, out_dist, out_ld, lk);
}

extern "C" int apsp_server_stats(apsp_server *h, apsp_stats *out, int reset) {
  if (!h || !out) return APSP_EINVAL;
  Server *s = &h->s;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->queued = (int64_t)s->queue.size();
  out->inflight = s->inflight;
  out->bytes_resident = s->bytes_resident;
  if (!s->lat_ms.empty()) {
    std::vector<double> v = s->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (double)(v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
    const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
    out->graphs_per_s = span > 0 ? (double)v.size() / span : 0.0;
  }
  if (reset) {
    s->lat_ms.clear();
    s->submitted = s->completed = s->failed = 0;
    s->any = false;
  }
  return APSP_OK;
}

extern "C" int apsp_server_destroy(apsp_server *h) {
  if (!h) return APSP_EINVAL;
  Server *s = &h->s;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->sched.joinable()) s->sched.join();
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->cfg.device);
  for (auto st : s->streams) cudaStreamSynchronize(st);  // in-flight requests finish (callbacks run)
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &kv : s->table) {
      if (kv.second->host) cudaFreeHost(kv.second->host);
      delete kv.second;
    }
    s->table.clear();
    for (auto &kv : s->pinned_free) cudaFreeHost(kv.second);
    s->pinned_free.clear();
  }
  if (s->desc_dev) cudaFree(s->desc_dev);
  for (auto w : s->workspaces)
    if (w) cudaFree(w);
  for (auto st : s->streams) cudaStreamDestroy(st);
  cudaSetDevice(prev);
  delete h;
  return APSP_OK;
}
