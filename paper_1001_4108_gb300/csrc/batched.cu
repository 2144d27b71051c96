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

constexpr int kBS = 64;          // tile side = k-block depth inside a CTA
constexpr int kBLD = kBS + 4;    // padded shared-memory row stride
constexpr int kBThreads = 256;   // (kBS / 4)^2: a 4 x 4 register block per thread
constexpr size_t kBSmem = 3 * (size_t)kBS * kBLD * 4 + 4 * kBS * 4 + 16;

template <typename T>
struct TileIO {
  using C = typename Arith<T>::C;
  // 4 x 4 block of tile (r0, c0) owned by (ty, tx): rows r0+4ty+a, cols c0+4tx+c
  __device__ static void load(const T *d, int64_t ld, int64_t n, int64_t r0, int64_t c0, int ty, int tx,
                              C (&x)[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gi = r0 + 4 * ty + a, gj = c0 + 4 * tx + c;
        x[a][c] = (gi < n && gj < n) ? Arith<T>::load(d[gi * ld + gj]) : Arith<T>::inf();
      }
  }
  __device__ static void store(T *d, int64_t ld, int64_t n, int64_t r0, int64_t c0, int ty, int tx,
                               const C (&x)[4][4], bool last) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gi = r0 + 4 * ty + a, gj = c0 + 4 * tx + c;
        if (gi < n && gj < n) d[gi * ld + gj] = last ? Arith<T>::finish(x[a][c]) : (T)x[a][c];
      }
  }
  __device__ static void to_smem(C *s, int ty, int tx, const C (&x)[4][4]) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) s[(4 * ty + a) * kBLD + 4 * tx + c] = x[a][c];
  }
};

// acc[a][c] <- min(acc[a][c], min_k A[4ty+a][k] + B[k][4tx+c]) over the tile's
// k's; A and B row-major in shared memory with stride kBLD.
template <typename T>
__device__ __forceinline__ void minplus_tile(typename Arith<T>::C (&acc)[4][4], const typename Arith<T>::C *A,
                                             const typename Arith<T>::C *B, int ty, int tx) {
  using C = typename Arith<T>::C;
#pragma unroll 4
  for (int kq = 0; kq < kBS / 4; ++kq) {
    C av[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const C *p = A + (4 * ty + a) * kBLD + 4 * kq;
      av[a][0] = p[0]; av[a][1] = p[1]; av[a][2] = p[2]; av[a][3] = p[3];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const C *q = B + (4 * kq + u) * kBLD + 4 * tx;
      const C bv[4] = {q[0], q[1], q[2], q[3]};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = Arith<T>::relax(acc[a][c], av[a][u], bv[c]);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kBThreads) fw_batched_cta(const BatchDesc *__restrict__ descs, int count,
                                                            int *counter) {
  using C = typename Arith<T>::C;
  using IO = TileIO<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *Ds = reinterpret_cast<C *>(smem_raw);  // closed diagonal tile
  C *Ps = Ds + kBS * kBLD;                  // first operand tile
  C *Qs = Ps + kBS * kBLD;                  // second operand tile
  C *rowbuf = Qs + kBS * kBLD;              // [2][kBS]
  C *colbuf = rowbuf + 2 * kBS;             // [2][kBS]
  int *s_g = reinterpret_cast<int *>(colbuf + 2 * kBS);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;

  while (true) {
    if (threadIdx.x == 0) *s_g = atomicAdd(counter, 1);
    __syncthreads();
    const int g = *s_g;
    __syncthreads();
    if (g >= count) return;
    T *d = static_cast<T *>(descs[g].d);
    const int64_t n = descs[g].n, ld = descs[g].ld;
    const int R = (int)((n + kBS - 1) / kBS);

    for (int b = 0; b < R; ++b) {
      const bool last = b == R - 1;
      const int64_t p0 = (int64_t)b * kBS;
      // ---- phase 1: close the diagonal tile (registers + row/column k broadcast)
      C x[4][4];
      IO::load(d, ld, n, p0, p0, ty, tx, x);
      if (ty == 0)
#pragma unroll
        for (int c = 0; c < 4; ++c) rowbuf[4 * tx + c] = x[0][c];
      if (tx == 0)
#pragma unroll
        for (int a = 0; a < 4; ++a) colbuf[4 * ty + a] = x[a][0];
      for (int kq = 0; kq < kBS / 4; ++kq) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = 4 * kq + u;
          __syncthreads();
          C rk[4], ck[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) rk[c] = rowbuf[(k & 1) * kBS + 4 * tx + c];
#pragma unroll
          for (int a = 0; a < 4; ++a) ck[a] = colbuf[(k & 1) * kBS + 4 * ty + a];
#pragma unroll
          for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) x[a][c] = Arith<T>::relax(x[a][c], ck[a], rk[c]);
          const int k1 = k + 1;
          if (k1 < kBS) {
            if (ty == (k1 >> 2))
#pragma unroll
              for (int c = 0; c < 4; ++c) rowbuf[(k1 & 1) * kBS + 4 * tx + c] = x[(u + 1) & 3][c];
            if (tx == (k1 >> 2))
#pragma unroll
              for (int a = 0; a < 4; ++a) colbuf[(k1 & 1) * kBS + 4 * ty + a] = x[a][(u + 1) & 3];
          }
        }
      }
      IO::store(d, ld, n, p0, p0, ty, tx, x, last);
      IO::to_smem(Ds, ty, tx, x);
      __syncthreads();
      // ---- phase 2: row panel D (x) X and column panel X (x) D
      for (int t = 0; t < 2 * (R - 1); ++t) {
        const bool row = t < R - 1;
        const int other = skip_pivot(row ? t : t - (R - 1), b);
        const int64_t r0 = row ? p0 : (int64_t)other * kBS, c0 = row ? (int64_t)other * kBS : p0;
        C acc[4][4];
        IO::load(d, ld, n, r0, c0, ty, tx, acc);
        IO::to_smem(Ps, ty, tx, acc);
        __syncthreads();
        if (row)
          minplus_tile<T>(acc, Ds, Ps, ty, tx);
        else
          minplus_tile<T>(acc, Ps, Ds, ty, tx);
        IO::store(d, ld, n, r0, c0, ty, tx, acc, last);
        __syncthreads();
      }
      // ---- phase 3: every other tile, A = column panel tile, B = row panel tile
      for (int ii = 0; ii < R - 1; ++ii) {
        const int64_t r0 = (int64_t)skip_pivot(ii, b) * kBS;
        C a[4][4];
        IO::load(d, ld, n, r0, p0, ty, tx, a);
        IO::to_smem(Ps, ty, tx, a);
        for (int jj = 0; jj < R - 1; ++jj) {
          const int64_t c0 = (int64_t)skip_pivot(jj, b) * kBS;
          C bt[4][4], acc[4][4];
          IO::load(d, ld, n, p0, c0, ty, tx, bt);
          IO::load(d, ld, n, r0, c0, ty, tx, acc);
          IO::to_smem(Qs, ty, tx, bt);
          __syncthreads();
          minplus_tile<T>(acc, Ps, Qs, ty, tx);
          IO::store(d, ld, n, r0, c0, ty, tx, acc, last);
          __syncthreads();
        }
      }
      __syncthreads();
    }
  }
}

template <typename T>
int launch_batched_kernel(const BatchDesc *descs, int count, int *counter, cudaStream_t st) {
  static thread_local int setup_mask = 0;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (!(setup_mask & (1 << (dev & 31)))) {
    if (cudaFuncSetAttribute(fw_batched_cta<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem) !=
        cudaSuccess)
      return APSP_ECUDA;
    setup_mask |= 1 << (dev & 31);
  }
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_batched_cta<T>, kBThreads, kBSmem) !=
      cudaSuccess)
    return APSP_ECUDA;
  const int grid = std::max(1, std::min(count, sms * std::max(per_sm, 1)));
  if (cudaMemsetAsync(counter, 0, sizeof(int), st) != cudaSuccess) return APSP_ECUDA;
  fw_batched_cta<T><<<grid, kBThreads, kBSmem, st>>>(descs, count, counter);
  return cudaPeekAtLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

}  // namespace

// Device buffer for the descriptors + work counter of each distinct batch,
// and a CUDA graph (counter reset + persistent kernel) once the same batch
// (same matrices, same stream) is solved a second time.
namespace {

struct BatchGraph {
  int dev;
  cudaStream_t stream;
  int dtype;
  std::vector<BatchDesc> descs;
  void *dev_buf = nullptr;  // descriptors followed by the counter
  cudaGraphExec_t exec = nullptr;
  int uses = 0;
};
std::mutex g_bmu;
std::vector<BatchGraph *> g_bgraphs;
constexpr size_t kMaxBatchGraphs = 8;

bool same_batch(const BatchGraph *e, const BatchDesc *d, int count, int dtype, cudaStream_t st, int dev) {
  if (e->dev != dev || e->stream != st || e->dtype != dtype || (int)e->descs.size() != count) return false;
  for (int i = 0; i < count; ++i)
    if (e->descs[i].d != d[i].d || e->descs[i].n != d[i].n || e->descs[i].ld != d[i].ld) return false;
  return true;
}

int launch_dtype(int dtype, const BatchDesc *descs, int count, int *counter, cudaStream_t st) {
  switch (dtype) {
    case APSP_I32: return launch_batched_kernel<int32_t>(descs, count, counter, st);
    case APSP_F32: return launch_batched_kernel<float>(descs, count, counter, st);
    case APSP_I16: return launch_batched_kernel<int16_t>(descs, count, counter, st);
  }
  return APSP_EINVAL;
}

}  // namespace

int run_batched_small(const BatchDesc *host_descs, int count, int dtype, cudaStream_t st, int dev) {
  if (count <= 0) return APSP_OK;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return APSP_ECUDA;
  if (cap != cudaStreamCaptureStatusNone) return APSP_EUNSUPPORTED;  // descriptors must be uploaded first
  std::lock_guard<std::mutex> lk(g_bmu);
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
    e = new BatchGraph{dev, st, dtype, std::vector<BatchDesc>(host_descs, host_descs + count)};
    const size_t bytes = (size_t)count * sizeof(BatchDesc) + 16;
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
  const BatchDesc *ddesc = static_cast<const BatchDesc *>(e->dev_buf);
  int *counter = reinterpret_cast<int *>(static_cast<char *>(e->dev_buf) + (size_t)count * sizeof(BatchDesc));
  ++e->uses;
  if (e->exec) return cudaGraphLaunch(e->exec, st) == cudaSuccess ? APSP_OK : APSP_ECUDA;
  if (e->uses < 2) return launch_dtype(dtype, ddesc, count, counter, st);
  // second use of the same batch: capture counter reset + persistent kernel
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return APSP_ECUDA;
  int rc = APSP_ECUDA;
  cudaGraph_t graph = nullptr;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const int lr = launch_dtype(dtype, ddesc, count, counter, cs);
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

}  // namespace apsp
