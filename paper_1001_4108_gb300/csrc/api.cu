// C ABI of libapsp (declared in include/apsp.h): argument checks, choice of
// the tile side, CUDA-graph replay of the stage loop, the host-buffer entry
// point and the device error word.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_internal.h"

// Device error word: bounded waits that give up record a code here.
static __device__ int g_apsp_err;
// Set by the negative-cycle check.
static __device__ int g_apsp_negcycle;

namespace apsp {

EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (EncodeTiledFn) nullptr;
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

namespace {

constexpr int kMaxDev = 64;

std::mutex g_mu;
int *g_err_ptr[kMaxDev];
int *g_neg_ptr[kMaxDev];

int elem_size(int dtype) { return dtype == APSP_I16 ? 2 : 4; }

// Device addresses of the error words for the current device (looked up once
// per device with that device current).
int device_words(int **err, int **neg) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return APSP_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_err_ptr[dev]) {
    void *pe = nullptr, *pn = nullptr;
    if (cudaGetSymbolAddress(&pe, g_apsp_err) != cudaSuccess) return APSP_ECUDA;
    if (cudaGetSymbolAddress(&pn, g_apsp_negcycle) != cudaSuccess) return APSP_ECUDA;
    g_err_ptr[dev] = static_cast<int *>(pe);
    g_neg_ptr[dev] = static_cast<int *>(pn);
  }
  *err = g_err_ptr[dev];
  if (neg) *neg = g_neg_ptr[dev];
  return APSP_OK;
}

// Tile side s: 64 keeps enough doubly dependent tiles in flight for small n,
// 128 halves the HBM traffic per relaxation (2 * elem / s bytes) for large n;
// the crossover comes from the tuning table (apsp_autotune).
int choose_kblock(int64_t n, int dtype, int32_t requested) {
  if (requested == 64 || requested == 128) return requested;
  return tuned_kblock(n, dtype);
}

int check_args(const void *dist, int64_t n, int64_t ld, int dtype, const apsp_options *opt) {
  if (dtype != APSP_I32 && dtype != APSP_F32 && dtype != APSP_I16) return APSP_EINVAL;
  if (n < 0 || ld < n || ld < 0) return APSP_EINVAL;
  if (n > (int64_t)1 << 20) return APSP_EUNSUPPORTED;  // grid and int index limits
  if (n > 0 && !dist) return APSP_EINVAL;
  if (opt) {
    if (opt->kblock != 0 && opt->kblock != 64 && opt->kblock != 128) return APSP_EINVAL;
    if (opt->events && opt->n_events < 0) return APSP_EINVAL;
  }
  return APSP_OK;
}

int run_dtype(const RunArgs &a, int dtype) {
  switch (dtype) {
    case APSP_I32: return run_i32(a);
    case APSP_F32: return run_f32(a);
    case APSP_I16: return run_i16(a);
  }
  return APSP_EINVAL;
}

// ------------------------------------------------------- lookahead streams
// One side stream (highest priority) and a fork / join event pair per
// (device, launching stream), created on first use outside of stream
// capture.  Work on one launching stream is ordered, so its solves can share
// them; a wait always refers to a record enqueued before it, so calls from
// several threads on one stream can only over-synchronise, never deadlock.
struct SideEntry {
  int dev;
  cudaStream_t stream;
  cudaStream_t side;
  cudaEvent_t fork, join;
  int prio;
};
constexpr size_t kMaxSide = 256;
std::vector<SideEntry> g_side;

// Fills a->side, fork, join, side_prio (nullptr side: no lookahead).  Caller
// holds g_mu.
void side_resources_locked(int dev, cudaStream_t stream, bool capturing, RunArgs *a) {
  a->side = nullptr;
  for (auto &e : g_side)
    if (e.dev == dev && e.stream == stream) {
      a->side = e.side;
      a->fork = e.fork;
      a->join = e.join;
      a->side_prio = e.prio;
      return;
    }
  // Never evicted (another thread may be enqueueing on an entry right now):
  // past kMaxSide launching streams, new ones run the plain schedule.
  if (capturing || g_side.size() >= kMaxSide) return;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return;
  SideEntry e{dev, stream, nullptr, nullptr, nullptr, greatest};
  if (cudaStreamCreateWithPriority(&e.side, cudaStreamNonBlocking, greatest) != cudaSuccess) return;
  if (cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming) != cudaSuccess) {
    if (e.fork) cudaEventDestroy(e.fork);
    cudaStreamDestroy(e.side);
    return;
  }
  g_side.push_back(e);
  a->side = e.side;
  a->fork = e.fork;
  a->join = e.join;
  a->side_prio = e.prio;
}

// ---------------------------------------------------------------- graphs
// A solve is 3 launches per stage (4 with the lookahead's split phase 3).
// Replaying them as one CUDA graph removes the per-launch host cost, which
// dominates for small n.  A graph is captured the
// second time the same (matrix, n, ld, dtype, s, flags) is solved, so one-off
// calls do not pay the instantiation.
struct GraphKey {
  void *d;
  int64_t n, ld;
  int dtype, S, flags, dev;
  cudaStream_t stream;
  void *ws;
  void *via;
  int64_t via_ld;
  const void *first_src;
  void *last_dst;
  bool operator==(const GraphKey &o) const {
    return d == o.d && n == o.n && ld == o.ld && dtype == o.dtype && S == o.S && flags == o.flags &&
           dev == o.dev && stream == o.stream && ws == o.ws && via == o.via && via_ld == o.via_ld &&
           first_src == o.first_src && last_dst == o.last_dst;
  }
};
struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec;
};
constexpr size_t kMaxGraphs = 32;
constexpr size_t kMaxSeen = 64;
std::vector<GraphEntry> g_graphs;
std::vector<GraphKey> g_seen;
cudaStream_t g_capture_stream[kMaxDev];

int launch_with_graph(const RunArgs &a, int dtype, int dev) {
  const GraphKey key{a.d, a.n, a.ld, dtype, a.S, a.flags, dev, a.stream, a.ws, a.via, a.via_ld, a.first_src,
                     a.last_dst};
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &g : g_graphs)
    if (g.key == key) return cudaGraphLaunch(g.exec, a.stream) == cudaSuccess ? APSP_OK : APSP_ECUDA;
  const bool seen = std::find(g_seen.begin(), g_seen.end(), key) != g_seen.end();
  if (!seen) {
    if (g_seen.size() >= kMaxSeen) g_seen.erase(g_seen.begin());
    g_seen.push_back(key);
    return run_dtype(a, dtype);
  }
  if (!g_capture_stream[dev] &&
      cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
    return APSP_ECUDA;
  RunArgs c = a;
  c.stream = g_capture_stream[dev];
  if (a.side) side_resources_locked(dev, c.stream, false, &c);
  if (cudaStreamBeginCapture(c.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return APSP_ECUDA;
  const int st = run_dtype(c, dtype);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c.stream, &graph);
  if (st != APSP_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return st != APSP_OK ? st : APSP_ECUDA;
  }
  cudaGraphExec_t exec = nullptr;
  // keep the side stream's launch priorities in the graph
  const cudaError_t ie = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return APSP_ECUDA;
  if (g_graphs.size() >= kMaxGraphs) {
    cudaGraphExecDestroy(g_graphs.front().exec);
    g_graphs.erase(g_graphs.begin());
  }
  g_graphs.push_back({key, exec});
  return cudaGraphLaunch(exec, a.stream) == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

// Library-owned workspaces, one per (device, stream): work on one stream is
// ordered, so a stream's solves can share one buffer.  Allocated outside of
// stream capture only; grown on demand.
struct WsEntry {
  int dev;
  cudaStream_t stream;
  void *p;
  size_t bytes;
};
constexpr size_t kMaxWs = 16;
std::vector<WsEntry> g_ws;

// Graphs captured with a workspace bake its address in: drop them before the
// buffer is freed.  Caller holds g_mu.
void forget_graphs_using(void *ws) {
  for (size_t i = 0; i < g_graphs.size();) {
    if (g_graphs[i].key.ws == ws) {
      cudaGraphExecDestroy(g_graphs[i].exec);
      g_graphs.erase(g_graphs.begin() + i);
    } else {
      ++i;
    }
  }
  g_seen.erase(std::remove_if(g_seen.begin(), g_seen.end(), [&](const GraphKey &k) { return k.ws == ws; }),
               g_seen.end());
}

void *library_workspace(int dev, cudaStream_t stream, size_t bytes, bool capturing, size_t *got) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &e : g_ws)
    if (e.dev == dev && e.stream == stream) {
      if (e.bytes >= bytes) {
        *got = e.bytes;
        return e.p;
      }
      if (capturing) return nullptr;
      cudaDeviceSynchronize();
      forget_graphs_using(e.p);
      cudaFree(e.p);
      e.p = nullptr;
      e.bytes = 0;
      if (cudaMalloc(&e.p, bytes) != cudaSuccess) return nullptr;
      e.bytes = bytes;
      *got = bytes;
      return e.p;
    }
  if (capturing) return nullptr;
  if (g_ws.size() >= kMaxWs) {
    cudaDeviceSynchronize();
    forget_graphs_using(g_ws.front().p);
    cudaFree(g_ws.front().p);
    g_ws.erase(g_ws.begin());
  }
  void *p = nullptr;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  g_ws.push_back({dev, stream, p, bytes});
  *got = bytes;
  return p;
}

// One panel copy (fp32 interleaved row panel, int16 replicated column panel).
size_t panel_bytes_for(int64_t n, int dtype, int S) {
  if (n <= S) return 0;
  if (dtype == APSP_F32) return interleaved_panel_bytes(n, S);
  if (dtype == APSP_I16) return replicated_panel_bytes(n, S);
  return 0;
}

// One panel buffer, two when the lookahead schedule applies (phase 2 of the
// next stage writes its copy while phase 3 reads the current one).
size_t workspace_bytes_for(int64_t n, int dtype, int S) {
  const size_t bufs = (n + S - 1) / S >= kLookaheadMinRounds ? 2 : 1;
  return bufs * panel_bytes_for(n, dtype, S);
}

// The workspace a call with `flags` uses: with APSP_FLAG_ONE_LAUNCH on a
// small matrix, at least the one-launch schedule's per-tile flags.
size_t workspace_bytes_with(int64_t n, int dtype, int S, int flags) {
  size_t bytes = workspace_bytes_for(n, dtype, S);
  const int64_t R = (n + S - 1) / S;
  if ((flags & APSP_FLAG_ONE_LAUNCH) && S == 64 && R >= kDataflowMinRounds && R <= kDataflowMaxRounds)
    bytes = std::max(bytes, dataflow_flag_bytes((int)R));
  return bytes;
}

// Device buffer of apsp_fw_host, one per device, grown on demand.
struct HostStage {
  std::mutex mu;
  void *buf = nullptr;
  size_t bytes = 0;
};
HostStage g_host_stage[kMaxDev];

}  // namespace

int default_kblock(int64_t n, int dtype) { return choose_kblock(n, dtype, 0); }
int error_word(int **err) { return device_words(err, nullptr); }

}  // namespace apsp

using namespace apsp;

extern "C" const char *apsp_status_str(int s) {
  switch (s) {
    case APSP_OK: return "APSP_OK";
    case APSP_EINVAL: return "APSP_EINVAL";
    case APSP_ENOMEM: return "APSP_ENOMEM";
    case APSP_EUNSUPPORTED: return "APSP_EUNSUPPORTED";
    case APSP_ECUDA: return "APSP_ECUDA";
    case APSP_ETIMEOUT: return "APSP_ETIMEOUT";
    case APSP_EBUSY: return "APSP_EBUSY";
    case APSP_EPENDING: return "APSP_EPENDING";
    case APSP_ENEGCYCLE: return "APSP_ENEGCYCLE";
  }
  return "APSP_UNKNOWN";
}

extern "C" int apsp_version(void) { return 100; }

extern "C" int64_t apsp_workspace_bytes(int64_t n, int dtype, int32_t kblock) {
  if (n < 0 || (dtype != APSP_I32 && dtype != APSP_F32 && dtype != APSP_I16)) return 0;
  return (int64_t)workspace_bytes_for(n, dtype, choose_kblock(n, dtype, kblock));
}

extern "C" int apsp_query_config(int64_t n, int dtype, int32_t kblock, apsp_config *cfg) {
  if (!cfg || n < 0 || (dtype != APSP_I32 && dtype != APSP_F32 && dtype != APSP_I16)) return APSP_EINVAL;
  if (kblock != 0 && kblock != 64 && kblock != 128) return APSP_EINVAL;
  const int S = choose_kblock(n, dtype, kblock);
  cfg->kblock = S;
  cfg->rounds = (int32_t)((n + S - 1) / S);
  cfg->phase3_tma = 1;
  cfg->phase3_threads = (S / 8) * (S / 8);
  const int64_t m = std::max<int64_t>(n - S, 0);
  cfg->phase3_relax_per_round = m * m * S;
  cfg->lookahead = cfg->rounds >= kLookaheadMinRounds ? 1 : 0;
  cfg->strips = uses_strips(S, cfg->rounds, dtype == APSP_F32, dtype == APSP_I16) ? 1 : 0;
  return APSP_OK;
}

namespace apsp {
namespace {
// apsp_fw_ex, optionally with the path bookkeeping of apsp_fw_paths.
int solve(void *dist, int64_t n, int64_t ld, int dtype, const apsp_options *opt, void *stream, int16_t *via,
          int64_t via_ld, const void *first_src = nullptr, int64_t first_src_ld = 0, void *last_dst = nullptr,
          int64_t last_dst_ld = 0) {
  int st = check_args(dist, n, ld, dtype, opt);
  if (st != APSP_OK) return st;
  if (n == 0) return APSP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDev) return APSP_ECUDA;
  int *err = nullptr, *neg = nullptr;
  st = device_words(&err, &neg);
  if (st != APSP_OK) return st;

  RunArgs a{};
  a.d = dist;
  a.n = n;
  a.ld = ld;
  a.S = choose_kblock(n, dtype, opt ? opt->kblock : 0);
  a.flags = opt ? opt->flags : 0;
  a.events = opt ? opt->events : nullptr;
  a.n_events = opt ? opt->n_events : 0;
  a.stream = static_cast<cudaStream_t>(stream);
  a.err = err;
  a.via = via;
  a.via_ld = via_ld;
  a.first_src = first_src;
  a.first_src_ld = first_src_ld;
  a.last_dst = last_dst;
  a.last_dst_ld = last_dst_ld;
  const size_t es = (size_t)elem_size(dtype);
  a.tma_ok = (reinterpret_cast<uintptr_t>(dist) % 16 == 0) && ((size_t)ld * es) % 16 == 0;

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(a.stream, &cap) != cudaSuccess) return APSP_ECUDA;
  if (cap != cudaStreamCaptureStatusNone && (a.flags & (APSP_FLAG_VALIDATE | APSP_FLAG_NEGCYCLE)))
    return APSP_EINVAL;  // both synchronize the stream
  const bool narrow = dtype == APSP_I32 && (a.flags & APSP_FLAG_NARROW);
  if (narrow && (via || (opt && opt->workspace))) return APSP_EINVAL;
  if (a.flags & APSP_FLAG_VALIDATE) {
    st = validate_input(dist, n, ld, dtype, a.stream, narrow);
    if (st != APSP_OK) return st;
  }
  if (narrow) {
    // int32 in and out, solved as int16x2 in a library buffer:
    // [n x ld16 int16 copy][int16 panel workspace]
    const int64_t ld16 = (n + 7) / 8 * 8;
    const int S16 = choose_kblock(n, APSP_I16, opt ? opt->kblock : 0);
    const size_t copy_bytes = ((size_t)n * ld16 * 2 + 255) / 256 * 256;
    const size_t ws16 = workspace_bytes_for(n, APSP_I16, S16);
    size_t got = 0;
    char *buf = static_cast<char *>(
        library_workspace(dev, a.stream, copy_bytes + ws16, cap != cudaStreamCaptureStatusNone, &got));
    if (buf) {  // else (first use inside a capture): the int32 path, same result
      if (narrow_to_i16(static_cast<const int32_t *>(dist), n, ld, reinterpret_cast<int16_t *>(buf), ld16,
                        a.stream) != APSP_OK)
        return APSP_ECUDA;
      RunArgs b = a;
      b.d = buf;
      b.ld = ld16;
      b.S = S16;
      b.tma_ok = true;  // 256-byte aligned buffer, 16-byte rows
      b.ws = ws16 ? buf + copy_bytes : nullptr;
      b.ws_bytes = ws16 ? got - copy_bytes : 0;
      if (!(b.flags & APSP_FLAG_NO_LOOKAHEAD)) {
        std::lock_guard<std::mutex> lk(g_mu);
        side_resources_locked(dev, b.stream, cap != cudaStreamCaptureStatusNone, &b);
      }
      const bool direct = (b.flags & APSP_FLAG_NO_GRAPH) || b.events || cap != cudaStreamCaptureStatusNone;
      st = direct ? run_dtype(b, APSP_I16) : launch_with_graph(b, APSP_I16, dev);
      if (st != APSP_OK) return st;
      if (widen_from_i16(reinterpret_cast<const int16_t *>(buf), ld16, n, static_cast<int32_t *>(dist), ld,
                         a.stream) != APSP_OK)
        return APSP_ECUDA;
      if (a.flags & APSP_FLAG_NEGCYCLE) return check_negcycle(dist, n, ld, dtype, a.stream, neg);
      return APSP_OK;
    }
  }
  const size_t need = (a.flags & APSP_FLAG_NO_WORKSPACE) ? 0 : workspace_bytes_with(n, dtype, a.S, a.flags);
  if (need) {
    if (opt && opt->workspace) {
      // one panel buffer is enough (plain schedule); two allow the lookahead
      if (opt->workspace_bytes < (int64_t)panel_bytes_for(n, dtype, a.S) ||
          reinterpret_cast<uintptr_t>(opt->workspace) % 256)
        return APSP_EINVAL;
      a.ws = opt->workspace;
      a.ws_bytes = (size_t)opt->workspace_bytes;
    } else {
      a.ws = library_workspace(dev, a.stream, need, cap != cudaStreamCaptureStatusNone, &a.ws_bytes);
      if (!a.ws) a.ws_bytes = 0;  // the kernels fall back to the form that needs none
    }
  }
  if (!(a.flags & APSP_FLAG_NO_LOOKAHEAD)) {
    std::lock_guard<std::mutex> lk(g_mu);
    side_resources_locked(dev, a.stream, cap != cudaStreamCaptureStatusNone, &a);
  }
  if (via && cudaMemset2DAsync(via, (size_t)via_ld * sizeof(int16_t), 0xff, (size_t)n * sizeof(int16_t), (size_t)n,
                               a.stream) != cudaSuccess)  // every entry -1: never improved
    return APSP_ECUDA;
  const bool direct = (a.flags & APSP_FLAG_NO_GRAPH) || a.events || cap != cudaStreamCaptureStatusNone;
  st = direct ? run_dtype(a, dtype) : launch_with_graph(a, dtype, dev);
  if (st != APSP_OK) return st;
  if (a.flags & APSP_FLAG_NEGCYCLE) return check_negcycle(dist, n, ld, dtype, a.stream, neg);
  return APSP_OK;
}
}  // namespace
}  // namespace apsp

extern "C" int apsp_fw_ex(void *dist, int64_t n, int64_t ld, int dtype, const apsp_options *opt, void *stream) {
  return solve(dist, n, ld, dtype, opt, stream, nullptr, 0);
}

extern "C" int apsp_fw_paths(void *dist, int16_t *via, int64_t n, int64_t ld, int64_t via_ld, int dtype,
                             const apsp_options *opt, void *stream) {
  const int st = check_args(dist, n, ld, dtype, opt);
  if (st != APSP_OK) return st;
  if (n > 0 && (!via || via_ld < n)) return APSP_EINVAL;
  const int S = choose_kblock(n, dtype, opt ? opt->kblock : 0);
  if ((n + S - 1) / S > 32767) return APSP_EUNSUPPORTED;  // stage numbers must fit int16
  return solve(dist, n, ld, dtype, opt, stream, via, via_ld);
}

extern "C" int apsp_fw(void *dist, int64_t n, int64_t ld, int dtype, void *stream) {
  return apsp_fw_ex(dist, n, ld, dtype, nullptr, stream);
}

extern "C" int apsp_fw_batched(void *const *dists, const int64_t *ns, const int64_t *lds, int64_t count, int dtype,
                               void *stream) {
  if (count < 0 || (count > 0 && (!dists || !ns || !lds))) return APSP_EINVAL;
  if (count > (int64_t)1 << 30) return APSP_EUNSUPPORTED;
  for (int64_t g = 0; g < count; ++g) {
    const int st = check_args(dists[g], ns[g], lds[g], dtype, nullptr);
    if (st != APSP_OK) return st;
  }
  if (count == 0) return APSP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDev) return APSP_ECUDA;
  // largest first: the persistent CTAs finish together
  std::vector<int64_t> order((size_t)count);
  for (int64_t g = 0; g < count; ++g) order[(size_t)g] = g;
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return ns[x] > ns[y]; });
  std::vector<BatchDesc> small;
  small.reserve((size_t)count);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int64_t g : order) {
    if (ns[g] == 0) continue;
    if (ns[g] > kBatchCtaMaxN) {
      const int st = apsp_fw_ex(dists[g], ns[g], lds[g], dtype, nullptr, stream);
      if (st != APSP_OK) return st;
    } else {
      small.push_back({dists[g], lds[g], ns[g]});
    }
  }
  return run_batched_small(small.data(), (int)small.size(), dtype, s, dev);
}

extern "C" int apsp_fw_host(void *host_dist, int64_t n, int64_t ld, int dtype, void *stream) {
  int st = check_args(host_dist, n, ld, dtype, nullptr);
  if (st != APSP_OK) return st;
  if (n == 0) return APSP_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev >= kMaxDev) return APSP_ECUDA;
  const size_t es = (size_t)elem_size(dtype);
  const int64_t dld = (n + 7) / 8 * 8;  // 16-byte aligned device rows
  const size_t bytes = (size_t)n * dld * es;
  HostStage &hs = g_host_stage[dev];
  std::lock_guard<std::mutex> lk(hs.mu);
  if (hs.bytes < bytes) {
    if (hs.buf) {
      cudaDeviceSynchronize();
      cudaFree(hs.buf);
      hs.buf = nullptr;
      hs.bytes = 0;
    }
    if (cudaMalloc(&hs.buf, bytes) != cudaSuccess) return APSP_ENOMEM;
    hs.bytes = bytes;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t row = (size_t)n * es, hpitch = (size_t)ld * es, dpitch = (size_t)dld * es;
  char *hb = static_cast<char *>(host_dist), *db = static_cast<char *>(hs.buf);
  // Pinned (device-mapped) host memory: the first stage's phase 3 reads its
  // tiles from it and the last stage's phase 3 writes them back, so only the
  // first stage's panels go in and the last stage's panels come out as
  // copies.  Otherwise: the whole matrix each way.
  const int S = choose_kblock(n, dtype, 0);
  cudaPointerAttributes pa{};
  const bool mapped = cudaPointerGetAttributes(&pa, host_dist) == cudaSuccess &&
                      pa.type == cudaMemoryTypeHost && pa.devicePointer != nullptr;
  // the kernels move C rows in 16-byte vectors: 16-byte aligned rows only
  const bool aligned = reinterpret_cast<uintptr_t>(pa.devicePointer) % 16 == 0 && hpitch % 16 == 0;
  if (mapped && aligned && (dtype == APSP_F32 || dtype == APSP_I32) && n % S == 0 && n > S) {
    const int64_t pb = n - S;  // first row / column of the last block
    cudaError_t e = cudaMemcpy2DAsync(db, dpitch, hb, hpitch, row, S, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(db + S * dpitch, dpitch, hb + S * hpitch, hpitch, S * es, n - S,
                            cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return APSP_ECUDA;
    st = solve(hs.buf, n, dld, dtype, nullptr, stream, nullptr, 0, pa.devicePointer, ld, pa.devicePointer, ld);
    if (st == APSP_OK) {
      e = cudaMemcpy2DAsync(hb + pb * hpitch, hpitch, db + pb * dpitch, dpitch, row, S, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(hb + pb * es, hpitch, db + pb * es, dpitch, S * es, pb, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return APSP_ECUDA;
      return cudaStreamSynchronize(s) == cudaSuccess ? APSP_OK : APSP_ECUDA;
    }
    if (st != APSP_EUNSUPPORTED) return st;  // else: the copying form below
  }
  // one linear copy each way when the rows are contiguous on both sides (a
  // pitched copy of n rows moves the same bytes at a fraction of the rate)
  const bool linear = ld == dld;
  cudaError_t e = linear ? cudaMemcpyAsync(hs.buf, host_dist, bytes, cudaMemcpyHostToDevice, s)
                         : cudaMemcpy2DAsync(hs.buf, dpitch, host_dist, hpitch, row, n, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return APSP_ECUDA;
  st = apsp_fw_ex(hs.buf, n, dld, dtype, nullptr, stream);
  if (st != APSP_OK) return st;
  e = linear ? cudaMemcpyAsync(host_dist, hs.buf, bytes, cudaMemcpyDeviceToHost, s)
             : cudaMemcpy2DAsync(host_dist, hpitch, hs.buf, dpitch, row, n, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return APSP_ECUDA;
  return cudaStreamSynchronize(s) == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

extern "C" int apsp_device_error(int reset) {
  int *err = nullptr;
  if (device_words(&err, nullptr) != APSP_OK) return -1;
  if (cudaDeviceSynchronize() != cudaSuccess) return -1;
  int h = 0;
  if (cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
  if (reset && h && cudaMemset(err, 0, sizeof(int)) != cudaSuccess) return -1;
  return h;
}
