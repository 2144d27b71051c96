// Batched all-pairs shortest paths: many independent graphs in one persistent
// launch.  Each CTA takes the next graph from a work counter (largest first)
// and runs every stage of Fig. 2 for it itself -- phase 1 on the diagonal
// tile in registers, phases 2 and 3 as min-plus tile products staged in
// shared memory, one __syncthreads between dependent steps -- so no launch or
// inter-CTA synchronization separates the stages of a small graph.
// Graphs above the size limit of one CTA are solved with the multi-CTA path.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/apsp.h"
#include "apsp_common.cuh"
#include "apsp_internal.h"
#include "cta_tile.cuh"

namespace apsp {

namespace {

template <typename T, int S, int M>
__global__ void __launch_bounds__(BShape<S, M>::NT, BShape<S, M>::MIN_BLOCKS)
    fw_batched_cta(const BatchDesc *__restrict__ descs, int count,
                                                                   int *counter) {
  using C = typename Arith<T>::C;
  using IO = TileIO<T, S, M>;
  constexpr int LD = BShape<S, M>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *Ds = reinterpret_cast<C *>(smem_raw);  // closed diagonal tile
  C *Ps = Ds + S * LD;                      // first operand tile
  C *Qs = Ps + S * LD;                      // second operand tile
  C *rowbuf = Qs + S * LD;                  // [2][2][S]
  C *colbuf = rowbuf + 4 * S;               // [2][2][S]
  int *s_g = reinterpret_cast<int *>(colbuf + 4 * S);
  int ty, tx;
  block_of_thread<S, M>(threadIdx.x, ty, tx);

  while (true) {
    if (threadIdx.x == 0) *s_g = atomicAdd(counter, 1);
    __syncthreads();
    const int g = *s_g;
    __syncthreads();
    if (g >= count) return;
    T *d = static_cast<T *>(descs[g].d);
    const int64_t n = descs[g].n, ld = descs[g].ld;
    const bool vec = IO::kVec && reinterpret_cast<uintptr_t>(d) % 16 == 0 && ld % 4 == 0;
    const int R = (int)((n + S - 1) / S);

    for (int b = 0; b < R; ++b) {
      const bool last = b == R - 1;
      const int64_t p0 = (int64_t)b * S;
      const int kvalid = (int)min((int64_t)S, n - p0);  // vertices of k-block b inside the graph
      const int kq_end = (kvalid + 3) / 4;
      // ---- phase 1: close the diagonal tile (registers + row/column k broadcast)
      close_diag<T, S, M>(d, ld, n, p0, kvalid, last, vec, Ds, rowbuf, colbuf, ty, tx);
      // ---- phase 2: row panel D (x) X and column panel X (x) D
      for (int t = 0; t < 2 * (R - 1); ++t) {
        const bool row = t < R - 1;
        const int other = skip_pivot(row ? t : t - (R - 1), b);
        const int64_t r0 = row ? p0 : (int64_t)other * S, c0 = row ? (int64_t)other * S : p0;
        C acc[M][M];
        IO::load(d, ld, n, r0, c0, ty, tx, acc, vec);
        IO::to_smem(Ps, ty, tx, acc);
        __syncthreads();
        if (warp_has_work<M>(ty, tx, (int)min((int64_t)S, n - r0), (int)min((int64_t)S, n - c0))) {
          if (row)
            minplus_tile<T, S, M>(acc, Ds, Ps, ty, tx, kq_end);
          else
            minplus_tile<T, S, M>(acc, Ps, Ds, ty, tx, kq_end);
        }
        IO::store(d, ld, n, r0, c0, ty, tx, acc, last, vec);
        __syncthreads();
      }
      // ---- phase 3: every other tile, A = column panel tile, B = row panel tile
      for (int ii = 0; ii < R - 1; ++ii) {
        const int64_t r0 = (int64_t)skip_pivot(ii, b) * S;
        C a[M][M];
        IO::load(d, ld, n, r0, p0, ty, tx, a, vec);
        IO::to_smem(Ps, ty, tx, a);
        for (int jj = 0; jj < R - 1; ++jj) {
          const int64_t c0 = (int64_t)skip_pivot(jj, b) * S;
          C bt[M][M], acc[M][M];
          IO::load(d, ld, n, p0, c0, ty, tx, bt, vec);
          IO::load(d, ld, n, r0, c0, ty, tx, acc, vec);
          IO::to_smem(Qs, ty, tx, bt);
          __syncthreads();
          if (warp_has_work<M>(ty, tx, (int)min((int64_t)S, n - r0), (int)min((int64_t)S, n - c0)))
            minplus_tile<T, S, M>(acc, Ps, Qs, ty, tx, kq_end);
          IO::store(d, ld, n, r0, c0, ty, tx, acc, last, vec);
          __syncthreads();
        }
      }
      __syncthreads();
    }
  }
}

template <typename T, int S, int M>
int launch_batched_kernel(const BatchDesc *descs, int count, int *counter, cudaStream_t st) {
  using B = BShape<S, M>;
  static thread_local uint64_t setup_mask = 0;  // bit per device
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APSP_ECUDA;
  if (!(setup_mask & (1ull << dev))) {
    if (cudaFuncSetAttribute(fw_batched_cta<T, S, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM) !=
        cudaSuccess)
      return APSP_ECUDA;
    setup_mask |= 1ull << dev;
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batched_cta<T, S, M>, B::NT, B::SMEM) !=
      cudaSuccess)
    return APSP_ECUDA;
  const int grid = std::max(1, std::min(count, sms * std::max(per_sm, 1)));
  if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return APSP_ECUDA;
  fw_batched_cta<T, S, M><<<grid, B::NT, B::SMEM, st>>>(descs, count, counter);
  return cudaPeekAtLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

template <typename T>
int launch_variant(int variant, const BatchDesc *descs, int count, int *counter, cudaStream_t st) {
  switch (variant) {
    case 0: return launch_batched_kernel<T, 32, 2>(descs, count, counter, st);
    case 1: return launch_batched_kernel<T, 32, 4>(descs, count, counter, st);
    case 2: return launch_batched_kernel<T, 64, 4>(descs, count, counter, st);
    case 3: return launch_batched_kernel<T, 128, 4>(descs, count, counter, st);
  }
  return APSP_EINVAL;
}

}  // namespace

// Device buffer for the descriptors + work counters of each distinct batch,
// and a CUDA graph (counter resets + persistent kernels) once the same batch
// (same matrices, same stream) is solved a second time.  One kernel shape,
// one persistent launch, when a shape carries nearly all of the batch's work;
// else the graphs are grouped by the kernel shape the tuning table picks for
// their n (the descriptors are sorted by n, so each group is a contiguous
// range) and the groups run concurrently on forked streams, joined back on
// the caller's stream.
namespace {

struct Group {
  int variant, first, count;
};

struct BatchGraph {
  int dev;
  cudaStream_t stream;
  int dtype;
  std::vector<BatchDesc> descs;
  std::vector<Group> groups;
  void *dev_buf = nullptr;  // descriptors, then one 16-byte counter slot per group
  cudaGraphExec_t exec = nullptr;
  int uses = 0;
};
// share of a batch's work above which one kernel shape takes every graph
constexpr double kSingleLaunchShare = 0.95;
std::mutex g_bmu;
std::vector<BatchGraph *> g_bgraphs;
constexpr size_t kMaxBatchGraphs = 8;
constexpr int kMaxGroups = 4;
cudaStream_t g_fork[64][kMaxGroups];
cudaEvent_t g_fork_ev[64][kMaxGroups + 1];

bool same_batch(const BatchGraph *e, const BatchDesc *d, int count, int dtype, cudaStream_t st, int dev) {
  if (e->dev != dev || e->stream != st || e->dtype != dtype || (int)e->descs.size() != count) return false;
  for (int i = 0; i < count; ++i)
    if (e->descs[i].d != d[i].d || e->descs[i].n != d[i].n || e->descs[i].ld != d[i].ld) return false;
  return true;
}

int launch_dtype(int dtype, int variant, const BatchDesc *descs, int count, int *counter, cudaStream_t st) {
  switch (dtype) {
    case APSP_I32: return launch_variant<int32_t>(variant, descs, count, counter, st);
    case APSP_F32: return launch_variant<float>(variant, descs, count, counter, st);
    case APSP_I16: return launch_variant<int16_t>(variant, descs, count, counter, st);
  }
  return APSP_EINVAL;
}

int fork_resources(int dev) {
  if (g_fork_ev[dev][0]) return APSP_OK;
  for (int i = 0; i < kMaxGroups; ++i)
    if (cudaStreamCreateWithFlags(&g_fork[dev][i], cudaStreamNonBlocking) != cudaSuccess) return APSP_ECUDA;
  for (int i = 0; i <= kMaxGroups; ++i)
    if (cudaEventCreateWithFlags(&g_fork_ev[dev][i], cudaEventDisableTiming) != cudaSuccess) return APSP_ECUDA;
  return APSP_OK;
}

// Enqueue all groups on `st` (one group inline, the others forked).
int enqueue_groups(const BatchGraph *e, cudaStream_t st) {
  const BatchDesc *ddesc = static_cast<const BatchDesc *>(e->dev_buf);
  char *ctr = static_cast<char *>(e->dev_buf) + e->descs.size() * sizeof(BatchDesc);
  const int ng = (int)e->groups.size();
  if (ng == 1) {
    const Group &g = e->groups[0];
    return launch_dtype(e->dtype, g.variant, ddesc + g.first, g.count, reinterpret_cast<int *>(ctr), st);
  }
  if (cudaEventRecord(g_fork_ev[e->dev][kMaxGroups], st) != cudaSuccess) return APSP_ECUDA;
  for (int i = 0; i < ng; ++i) {
    cudaStream_t s = g_fork[e->dev][i];
    if (cudaStreamWaitEvent(s, g_fork_ev[e->dev][kMaxGroups], 0) != cudaSuccess) return APSP_ECUDA;
    const Group &g = e->groups[i];
    const int rc = launch_dtype(e->dtype, g.variant, ddesc + g.first, g.count, reinterpret_cast<int *>(ctr + 16 * i), s);
    if (rc != APSP_OK) return rc;
    if (cudaEventRecord(g_fork_ev[e->dev][i], s) != cudaSuccess) return APSP_ECUDA;
    if (cudaStreamWaitEvent(st, g_fork_ev[e->dev][i], 0) != cudaSuccess) return APSP_ECUDA;
  }
  return APSP_OK;
}

}  // namespace

int run_batched_small(const BatchDesc *host_descs, int count, int dtype, cudaStream_t st, int dev) {
  if (count <= 0) return APSP_OK;
  if (dev < 0 || dev >= 64) return APSP_ECUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return APSP_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return APSP_EUNSUPPORTED;  // descriptors must be uploaded first
  std::lock_guard<std::mutex> lk(g_bmu);
  int rc = fork_resources(dev);
  if (rc != APSP_OK) return rc;
  BatchGraph *e = nullptr;
  for (auto *c : g_bgraphs)
    if (same_batch(c, host_descs, count, dtype, st, dev)) e = c;
  if (!e) {
    if (g_bgraphs.size() >= kMaxBatchGraphs) {
      BatchGraph *old = g_bgraphs.front();
      cudaDeviceSynchronize();
      if (old->exec) cudaGraphExecDestroy(old->exec);
      cudaFree(old->dev_buf);
      delete old;
      g_bgraphs.erase(g_bgraphs.begin());
    }
    e = new BatchGraph{dev, st, dtype, std::vector<BatchDesc>(host_descs, host_descs + count), {}};
    // One persistent launch for the whole batch when one kernel shape carries
    // nearly all of its work (sum of n^3): the graphs of the other shapes are
    // then few and small, and running them on that shape costs less than a
    // second launch (c4: 10.61 ms either way).  Otherwise one launch per
    // shape group, on forked streams.
    int single = -1;
    {
      double work[kBatchVariants] = {0}, total = 0;
      for (int i = 0; i < count; ++i) {
        const double w = (double)host_descs[i].n * host_descs[i].n * host_descs[i].n;
        work[tuned_batch_variant(host_descs[i].n, dtype)] += w;
        total += w;
      }
      for (int v = 0; v < kBatchVariants; ++v)
        if (work[v] >= kSingleLaunchShare * total) single = v;
    }
    for (int i = 0; i < count; ++i) {
      const int v = single >= 0 ? single : tuned_batch_variant(host_descs[i].n, dtype);
      if (e->groups.empty() || e->groups.back().variant != v) {
        if ((int)e->groups.size() == kMaxGroups) {  // merge the tail into the last group
          e->groups.back().count = count - e->groups.back().first;
          break;
        }
        e->groups.push_back({v, i, 0});
      }
      e->groups.back().count = i + 1 - e->groups.back().first;
    }
    const size_t bytes = (size_t)count * sizeof(BatchDesc) + 16 * kMaxGroups;
    if (cudaMalloc(&e->dev_buf, bytes) != cudaSuccess) {
      delete e;
      return APSP_ENOMEM;
    }
    if (cudaMemcpyAsync(e->dev_buf, e->descs.data(), (size_t)count * sizeof(BatchDesc), cudaMemcpyHostToDevice,
                        st) != cudaSuccess) {
      cudaFree(e->dev_buf);
      delete e;
      return APSP_ECUDA;
    }
    g_bgraphs.push_back(e);
  }
  ++e->uses;
  if (e->exec) return cudaGraphLaunch(e->exec, st) == cudaSuccess ? APSP_OK : APSP_ECUDA;
  if (e->uses < 2) return enqueue_groups(e, st);
  // second use of the same batch: capture the counter resets + kernels
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return APSP_ECUDA;
  rc = APSP_ECUDA;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const int lr = enqueue_groups(e, cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (lr == APSP_OK && ce == cudaSuccess && cudaGraphInstantiate(&e->exec, graph, 0) == cudaSuccess)
      rc = cudaGraphLaunch(e->exec, st) == cudaSuccess ? APSP_OK : APSP_ECUDA;
    else
      rc = lr != APSP_OK ? lr : APSP_ECUDA;
    if (graph) cudaGraphDestroy(graph);
  }
  cudaStreamDestroy(cs);
  return rc;
}

// Batched launch without caching (the serving loop's path): uploads the
// descriptors (sorted by n, largest first) into a device buffer grown in
// stream order, then launches one persistent kernel per kernel-shape group, in
// order, on `st`.
int run_batched_direct(const BatchDesc *host_descs, int count, int dtype, cudaStream_t st, void **dev_buf,
                       size_t *cap, bool match_single) {
  if (count <= 0) return APSP_OK;
  const size_t need = (size_t)count * sizeof(BatchDesc) + 16 * kBatchVariants * 2;
  if (*cap < need) {
    if (*dev_buf) cudaFreeAsync(*dev_buf, st);
    *dev_buf = nullptr;
    *cap = 0;
    size_t c = 4096;
    while (c < need) c <<= 1;
    if (cudaMallocAsync(dev_buf, c, st) != cudaSuccess) return APSP_ENOMEM;
    *cap = c;
  }
  // pageable source: the runtime stages it before returning
  if (cudaMemcpyAsync(*dev_buf, host_descs, (size_t)count * sizeof(BatchDesc), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return APSP_ECUDA;
  const BatchDesc *dd = static_cast<const BatchDesc *>(*dev_buf);
  char *ctr = static_cast<char *>(*dev_buf) + (size_t)count * sizeof(BatchDesc);
  auto variant_of = [&](int64_t n) {
    const int v = tuned_batch_variant(n, dtype);
    return match_single && n > 32 && v != 2 ? 2 : v;
  };
  int first = 0, slot = 0;
  while (first < count) {
    const int v = variant_of(host_descs[first].n);
    int last = first + 1;
    while (last < count && variant_of(host_descs[last].n) == v) ++last;
    const int rc = launch_dtype(dtype, v, dd + first, last - first, reinterpret_cast<int *>(ctr + 16 * slot), st);
    if (rc != APSP_OK) return rc;
    slot = (slot + 1) % (2 * kBatchVariants);
    first = last;
  }
  return APSP_OK;
}

// Times one kernel shape on `count` graphs (used by the autotuner).
int time_batched_variant(const BatchDesc *dev_descs, int count, int *counter, int dtype, int variant,
                         cudaStream_t st, float *ms) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return APSP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return APSP_ECUDA;
  }
  int rc = launch_dtype(dtype, variant, dev_descs, count, counter, st);  // warm-up
  if (rc == APSP_OK && cudaEventRecord(e0, st) != cudaSuccess) rc = APSP_ECUDA;
  if (rc == APSP_OK) rc = launch_dtype(dtype, variant, dev_descs, count, counter, st);
  if (rc == APSP_OK && cudaEventRecord(e1, st) != cudaSuccess) rc = APSP_ECUDA;
  if (rc == APSP_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess))
    rc = APSP_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

}  // namespace apsp
