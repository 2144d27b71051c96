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

namespace apsp {

namespace {

// Kernel shape: tile side S (= k-block depth inside the CTA) and an M x M
// register block per thread, (S/M)^2 threads; rows M*ty+a, columns M*tx+c.
template <int S, int M> struct BShape {
  static constexpr int Q = S / M;                 // threads per dimension
  static constexpr int NT = Q * Q;
  static constexpr int LD = S + 4;                // padded shared-memory row stride
  static constexpr size_t SMEM = 3 * (size_t)S * LD * 4 + 4 * (size_t)S * 4 + 16;
  // CTAs per SM the register budget is sized for (s 64: three, as the
  // shared memory allows; 0 = no bound)
  static constexpr int MIN_BLOCKS = S == 64 ? 3 : 0;
};

// Reinterprets a 32-bit word as the compute type (int32 or fp32).
template <typename C> __device__ __forceinline__ C word_as(int v);
template <> __device__ __forceinline__ int32_t word_as<int32_t>(int v) { return v; }
template <> __device__ __forceinline__ float word_as<float>(int v) { return __int_as_float(v); }

// Global <-> register moves of one S x S tile, M x M elements per thread
// (rows M ty + a, columns M tx + c).  `vec`: 32-bit elements, 16-byte
// aligned matrix and rows (ld % 4 == 0), so that with M = 4 each row of a
// thread's block moves as one 128-bit access.
template <typename T, int S, int M>
struct TileIO {
  using C = typename Arith<T>::C;
  static constexpr int LD = BShape<S, M>::LD;
  // A tile entirely inside the matrix needs no masks (the common case).
  static constexpr bool kVec = M == 4 && sizeof(T) == 4;
  __device__ static void load(const T *d, int64_t ld, int64_t n, int64_t r0, int64_t c0, int ty, int tx,
                              C (&x)[M][M], bool vec) {
    if (r0 + S <= n && c0 + S <= n) {
      const T *p = d + (r0 + M * ty) * ld + c0 + M * tx;
      if constexpr (kVec) {
        if (vec) {
#pragma unroll
          for (int a = 0; a < M; ++a) {
            const int4 v = *reinterpret_cast<const int4 *>(p + a * ld);
            x[a][0] = word_as<C>(v.x);
            x[a][1] = word_as<C>(v.y);
            x[a][2] = word_as<C>(v.z);
            x[a][3] = word_as<C>(v.w);
          }
          return;
        }
      }
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < M; ++c) x[a][c] = Arith<T>::load(p[a * ld + c]);
      return;
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const int64_t gi = r0 + M * ty + a, gj = c0 + M * tx + c;
        x[a][c] = (gi < n && gj < n) ? Arith<T>::load(d[gi * ld + gj]) : Arith<T>::inf();
      }
  }
  __device__ static void store(T *d, int64_t ld, int64_t n, int64_t r0, int64_t c0, int ty, int tx,
                               const C (&x)[M][M], bool last, bool vec) {
    if (r0 + S <= n && c0 + S <= n) {
      T *p = d + (r0 + M * ty) * ld + c0 + M * tx;
      if constexpr (kVec) {
        if (vec) {
#pragma unroll
          for (int a = 0; a < M; ++a) {
            C v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = last ? Arith<T>::finish(x[a][c]) : x[a][c];
            *reinterpret_cast<int4 *>(p + a * ld) =
                make_int4(__builtin_bit_cast(int, v[0]), __builtin_bit_cast(int, v[1]),
                          __builtin_bit_cast(int, v[2]), __builtin_bit_cast(int, v[3]));
          }
          return;
        }
      }
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < M; ++c) p[a * ld + c] = last ? Arith<T>::finish(x[a][c]) : (T)x[a][c];
      return;
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const int64_t gi = r0 + M * ty + a, gj = c0 + M * tx + c;
        if (gi < n && gj < n) d[gi * ld + gj] = last ? Arith<T>::finish(x[a][c]) : (T)x[a][c];
      }
  }
  __device__ static void to_smem(C *s, int ty, int tx, const C (&x)[M][M]) {
#pragma unroll
    for (int a = 0; a < M; ++a) {
      if constexpr (M == 4 && sizeof(C) == 4) {  // 16-byte aligned: padded rows of S + 4 words
        *reinterpret_cast<int4 *>(s + (M * ty + a) * LD + M * tx) =
            make_int4(__builtin_bit_cast(int, x[a][0]), __builtin_bit_cast(int, x[a][1]),
                      __builtin_bit_cast(int, x[a][2]), __builtin_bit_cast(int, x[a][3]));
      } else {
#pragma unroll
        for (int c = 0; c < M; ++c) s[(M * ty + a) * LD + M * tx + c] = x[a][c];
      }
    }
  }
};


// acc[a][c] <- min(acc[a][c], min_k A[M ty + a][k] + B[k][M tx + c]) over the
// first 4 * kq_end k's of the tile (the k-block's vertices inside the graph,
// rounded up: the padding k's hold infinity); A and B row-major in shared
// memory with the padded stride.
template <typename T, int S, int M>
__device__ __forceinline__ void minplus_tile(typename Arith<T>::C (&acc)[M][M], const typename Arith<T>::C *A,
                                             const typename Arith<T>::C *B, int ty, int tx, int kq_end) {
  using C = typename Arith<T>::C;
  constexpr int LD = BShape<S, M>::LD;
  static_assert(sizeof(C) == 4 && (M == 2 || M == 4), "vector shared loads of 4-byte elements");
  static_assert((LD * 4) % 16 == 0, "16-byte aligned rows");
#pragma unroll 4
  for (int kq = 0; kq < kq_end; ++kq) {
    C av[M][4];
#pragma unroll
    for (int a = 0; a < M; ++a) {  // 4 k's of row M ty + a: one 128-bit load
      const int4 v = *reinterpret_cast<const int4 *>(A + (M * ty + a) * LD + 4 * kq);
      av[a][0] = word_as<C>(v.x);
      av[a][1] = word_as<C>(v.y);
      av[a][2] = word_as<C>(v.z);
      av[a][3] = word_as<C>(v.w);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const C *q = B + (4 * kq + u) * LD + M * tx;
      C bv[M];
      if constexpr (M == 4) {
        const int4 v = *reinterpret_cast<const int4 *>(q);
        bv[0] = word_as<C>(v.x);
        bv[1] = word_as<C>(v.y);
        bv[2] = word_as<C>(v.z);
        bv[3] = word_as<C>(v.w);
      } else {
        const int2 v = *reinterpret_cast<const int2 *>(q);
        bv[0] = word_as<C>(v.x);
        bv[1] = word_as<C>(v.y);
      }
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < M; ++c) acc[a][c] = Arith<T>::relax(acc[a][c], av[a][u], bv[c]);
    }
  }
}

// Phase 1 inside one CTA: closes the diagonal tile (p0, p0) -- kvalid
// sequential k steps on an M x M register block per thread, row and column
// k + 1 published through a double buffer (one barrier per step) -- stores it
// (clamped in the last stage) and leaves it in Ds (padded rows).  Ends with a
// barrier.
template <typename T, int S, int M>
__device__ __forceinline__ void close_diag(T *d, int64_t ld, int64_t n, int64_t p0, int kvalid, bool last,
                                           bool vec, typename Arith<T>::C *Ds, typename Arith<T>::C *rowbuf,
                                           typename Arith<T>::C *colbuf, int ty, int tx) {
  using C = typename Arith<T>::C;
  using IO = TileIO<T, S, M>;
  C x[M][M];
  IO::load(d, ld, n, p0, p0, ty, tx, x, vec);
  if (ty == 0)
#pragma unroll
    for (int c = 0; c < M; ++c) rowbuf[M * tx + c] = x[0][c];
  if (tx == 0)
#pragma unroll
    for (int a = 0; a < M; ++a) colbuf[M * ty + a] = x[a][0];
  for (int kq = 0; kq < (kvalid + M - 1) / M; ++kq) {
#pragma unroll
    for (int u = 0; u < M; ++u) {
      const int k = M * kq + u;
      __syncthreads();
      C rk[M], ck[M];
#pragma unroll
      for (int c = 0; c < M; ++c) rk[c] = rowbuf[(k & 1) * S + M * tx + c];
#pragma unroll
      for (int a = 0; a < M; ++a) ck[a] = colbuf[(k & 1) * S + M * ty + a];
#pragma unroll
      for (int a = 0; a < M; ++a)
#pragma unroll
        for (int c = 0; c < M; ++c) x[a][c] = Arith<T>::relax(x[a][c], ck[a], rk[c]);
      const int k1 = k + 1;
      if (k1 < S) {
        if (ty == k1 / M)
#pragma unroll
          for (int c = 0; c < M; ++c) rowbuf[(k1 & 1) * S + M * tx + c] = x[(u + 1) % M][c];
        if (tx == k1 / M)
#pragma unroll
          for (int a = 0; a < M; ++a) colbuf[(k1 & 1) * S + M * ty + a] = x[a][(u + 1) % M];
      }
    }
  }
  IO::store(d, ld, n, p0, p0, ty, tx, x, last, vec);
  IO::to_smem(Ds, ty, tx, x);
  __syncthreads();
}

template <typename T, int S, int M>
__global__ void __launch_bounds__(BShape<S, M>::NT, BShape<S, M>::MIN_BLOCKS)
    fw_batched_cta(const BatchDesc *__restrict__ descs, int count,
                                                                   int *counter) {
  using C = typename Arith<T>::C;
  using IO = TileIO<T, S, M>;
  constexpr int Q = BShape<S, M>::Q;
  constexpr int LD = BShape<S, M>::LD;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *Ds = reinterpret_cast<C *>(smem_raw);  // closed diagonal tile
  C *Ps = Ds + S * LD;                      // first operand tile
  C *Qs = Ps + S * LD;                      // second operand tile
  C *rowbuf = Qs + S * LD;                  // [2][S]
  C *colbuf = rowbuf + 2 * S;               // [2][S]
  int *s_g = reinterpret_cast<int *>(colbuf + 2 * S);
  const int tx = threadIdx.x % Q, ty = threadIdx.x / Q;

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
        if (row)
          minplus_tile<T, S, M>(acc, Ds, Ps, ty, tx, kq_end);
        else
          minplus_tile<T, S, M>(acc, Ps, Ds, ty, tx, kq_end);
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
  static thread_local int setup_mask = 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (!(setup_mask & (1 << (dev & 31)))) {
    if (cudaFuncSetAttribute(fw_batched_cta<T, S, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B::SMEM) !=
        cudaSuccess)
      return APSP_ECUDA;
    setup_mask |= 1 << (dev & 31);
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
// (same matrices, same stream) is solved a second time.  Graphs are grouped
// by the kernel shape the tuning table picks for their n (the descriptors are
// sorted by n, so each group is a contiguous range); the groups run
// concurrently on forked streams and join back on the caller's stream.
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
    for (int i = 0; i < count; ++i) {
      const int v = tuned_batch_variant(host_descs[i].n, dtype);
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
