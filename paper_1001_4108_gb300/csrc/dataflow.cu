// Small matrices in one launch (APSP_FLAG_ONE_LAUNCH): every stage of Fig. 2
// for one matrix, its tiles spread over the CTAs of one cooperative launch,
// with the order of the stages kept by per-tile flags in global memory
// instead of launch boundaries.
//
// Below a few thousand vertices a stage is far too small to fill the GPU, and
// the multi-launch schedule is bound by its chain of dependent launches
// (phase 3 of the tiles of row and column b + 1, then phases 1 and 2 of stage
// b + 1).  Here each CTA owns a fixed set of tiles (tile t = I R + J belongs
// to CTA t mod grid) and walks the work of all stages in one global order,
// the order of the lookahead schedule:
//
//   phase 1, 2 of stage 0; then for b = 0 .. R-1:
//     cross(b)  phase 3 of stage b on the tiles of row and column b + 1,
//     phase 1 and phase 2 of stage b + 1,
//     rest(b)   phase 3 of stage b on the other tiles.
//
// Before a tile operation a CTA waits (one thread, acquire loads with a
// %globaltimer bound) for what it reads:
//   ver[I][J]  stages applied to tile (I, J): phase 2 of stage s waits for
//              ver[s][s] = s + 1, phase 3 for ver[I][s] = ver[s][J] = s + 1;
// and, before it overwrites a tile that was a panel in stage s - 1, for every
// stage-(s-1) reader of that panel to be done:
//   rd_row[b][J]  phase-3 tiles of stage b in column J done (readers of (b, J)),
//   rd_col[b][I]  phase-3 tiles of stage b in row I done (readers of (I, b)),
//   rd_diag[b]    phase-2 tiles of stage b done (readers of (b, b)).
// Every wait refers to work earlier in the global order, and all CTAs are
// resident (cooperative launch), so the earliest unfinished operation can
// always run: no deadlock.  A wait that runs out (2 s) or sees another CTA's
// error code records an error in the device error word and the CTA returns.
//
// Each tile operation is the one of the stage kernels at s = 64 (phase 1:
// k-sequential closure; phase 2: min-plus product with the closed diagonal
// tile; phase 3: min-plus product of the two panel tiles), with the same
// operations per element, so results equal the multi-launch schedule's bit
// for bit.
//
// Measured on a GB300 it is not faster than the multi-launch schedule
// (n = 1024 fp32: 333 us against 266 us; int32 about even up to n = 1536):
// the chain per stage -- the cross update of the next diagonal tile, its
// closure, the panel products, each a whole 64 x 64 tile on one SM, with a
// flag handoff between -- costs what the launch chain costs.  So it is
// opt-in.
#include <algorithm>

#include "../../include/apsp.h"
#include "apsp_common.cuh"
#include "apsp_internal.h"
#include "cta_tile.cuh"

namespace apsp {
namespace {

constexpr int kDS = 64, kDM = 4;  // tile side, register block per thread
using DShape = BShape<kDS, kDM>;  // 256 threads, padded shared rows
// Device error code of a dataflow wait that gave up (the TMA waits use 1).
constexpr int kDevTimeoutFlag = 2;

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int *p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(int *p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread: waits until *p >= v.  False if the wait ran out or another CTA
// has already recorded an error (then this CTA gives up too).
__device__ bool wait_geq(const int *p, int v, int *err) {
  if (ld_acquire(p) >= v) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (ld_acquire(p) >= v) return true;
    if (*reinterpret_cast<volatile int *>(err) != 0) return false;
    if (globaltimer_ns() - t0 > kWaitLimitNs) {
      atomicCAS(err, 0, kDevTimeoutFlag);
      return false;
    }
    __nanosleep(32);
  }
}

template <typename T>
__global__ void __launch_bounds__(DShape::NT, 2)
    fw_dataflow(T *__restrict__ d, int64_t n, int64_t ld, int R, int *flags, int *err) {
  using C = typename Arith<T>::C;
  using IO = TileIO<T, kDS, kDM, true>;  // loads through L2: tiles come from other SMs
  constexpr int S = kDS, M = kDM, LD = DShape::LD;
  __shared__ __align__(16) C As[S * LD];
  __shared__ __align__(16) C Bs[S * LD];
  __shared__ __align__(16) C rowbuf[4 * S];
  __shared__ __align__(16) C colbuf[4 * S];
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  int ty, tx;
  block_of_thread<kDS, kDM>(tid, ty, tx);
  int *ver = flags;             // [R * R]
  int *rd_row = ver + R * R;    // [R * R], index b * R + J
  int *rd_col = rd_row + R * R; // [R * R], index b * R + I
  int *rd_diag = rd_col + R * R;  // [R]
  const bool vec = IO::kVec && reinterpret_cast<uintptr_t>(d) % 16 == 0 && ld % 4 == 0;
  const int ntile = R * R;

  for (int step = -1; step < R; ++step) {
    const int b = step, b1 = step + 1;
    for (int cat = 0; cat < 4; ++cat) {
      for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int I = t / R, J = t % R;
        // the operation of tile t in (step, cat), if any: op 1, 2, 3 = phase
        int s = 0, op = 0;
        if (cat == 0) {  // cross(b)
          if (b >= 0 && b1 < R && I != b && J != b && (I == b1 || J == b1)) s = b, op = 3;
        } else if (cat == 1) {  // phase 1 of stage b + 1
          if (b1 < R && I == b1 && J == b1) s = b1, op = 1;
        } else if (cat == 2) {  // phase 2 of stage b + 1
          if (b1 < R && ((I == b1) != (J == b1))) s = b1, op = 2;
        } else {  // rest(b)
          if (b >= 0 && I != b && J != b && I != b1 && J != b1) s = b, op = 3;
        }
        if (op == 0) continue;

        if (tid == 0) {
          bool ok = true;
          if (op == 2) {
            ok = wait_geq(&ver[s * R + s], s + 1, err);
            if (ok && s >= 1 && I == s && J == s - 1) ok = wait_geq(&rd_col[(s - 1) * R + s], R - 1, err);
            if (ok && s >= 1 && J == s && I == s - 1) ok = wait_geq(&rd_row[(s - 1) * R + s], R - 1, err);
          } else if (op == 3) {
            ok = wait_geq(&ver[I * R + s], s + 1, err) && wait_geq(&ver[s * R + J], s + 1, err);
            if (ok && s >= 1) {
              if (I == s - 1 && J == s - 1) ok = wait_geq(&rd_diag[s - 1], 2 * (R - 1), err);
              else if (I == s - 1) ok = wait_geq(&rd_row[(s - 1) * R + J], R - 1, err);
              else if (J == s - 1) ok = wait_geq(&rd_col[(s - 1) * R + I], R - 1, err);
            }
          }
          s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;

        const int64_t p0 = (int64_t)s * S;
        const int kvalid = (int)min((int64_t)S, n - p0);
        const int kq_end = (kvalid + 3) / 4;
        const bool last = s == R - 1;
        const int64_t r0 = (int64_t)I * S, c0 = (int64_t)J * S;
        if (op == 1) {
          close_diag<T, S, M, true>(d, ld, n, p0, kvalid, last, vec, As, rowbuf, colbuf, ty, tx);
        } else if (op == 2) {
          C x[M][M], acc[M][M];
          IO::load(d, ld, n, p0, p0, ty, tx, x, vec);  // the closed diagonal tile
          IO::load(d, ld, n, r0, c0, ty, tx, acc, vec);
          IO::to_smem(As, ty, tx, x);
          IO::to_smem(Bs, ty, tx, acc);
          __syncthreads();
          if (warp_has_work<M>(ty, tx, (int)min((int64_t)S, n - r0), (int)min((int64_t)S, n - c0))) {
            if (I == s)
              minplus_tile<T, S, M>(acc, As, Bs, ty, tx, kq_end);  // row panel: D (x) X
            else
              minplus_tile<T, S, M>(acc, Bs, As, ty, tx, kq_end);  // column panel: X (x) D
          }
          IO::store(d, ld, n, r0, c0, ty, tx, acc, last, vec);
        } else {
          C a[M][M], bt[M][M], acc[M][M];
          IO::load(d, ld, n, r0, p0, ty, tx, a, vec);   // column-panel tile (I, s)
          IO::load(d, ld, n, p0, c0, ty, tx, bt, vec);  // row-panel tile (s, J)
          IO::load(d, ld, n, r0, c0, ty, tx, acc, vec);
          IO::to_smem(As, ty, tx, a);
          IO::to_smem(Bs, ty, tx, bt);
          __syncthreads();
          if (warp_has_work<M>(ty, tx, (int)min((int64_t)S, n - r0), (int)min((int64_t)S, n - c0)))
            minplus_tile<T, S, M>(acc, As, Bs, ty, tx, kq_end);
          IO::store(d, ld, n, r0, c0, ty, tx, acc, last, vec);
        }
        __syncthreads();  // the tile is stored and its operands read
        if (tid == 0) {
          __threadfence();
          st_release(&ver[t], s + 1);
          if (op == 2) red_release_add(&rd_diag[s], 1);
          if (op == 3) {
            red_release_add(&rd_row[s * R + J], 1);
            red_release_add(&rd_col[s * R + I], 1);
          }
        }
      }
    }
  }
}

template <typename T>
int launch_dataflow(const RunArgs &a, int *flags) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fw_dataflow<T>, DShape::NT, 0) != cudaSuccess ||
      per_sm < 1)
    return APSP_ECUDA;
  const int R = (int)((a.n + kDS - 1) / kDS);
  const int grid = std::min(R * R, sms * per_sm);
  if (cudaMemsetAsync(flags, 0, dataflow_flag_bytes(R), a.stream) != cudaSuccess) return APSP_ECUDA;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(DShape::NT);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = a.stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: the flag waits need it
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  T *d = static_cast<T *>(a.d);
  const cudaError_t e = cudaLaunchKernelEx(&cfg, fw_dataflow<T>, d, a.n, a.ld, R, flags, a.err);
  return e == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

}  // namespace

size_t dataflow_flag_bytes(int R) { return (size_t)(3 * R * R + R) * sizeof(int); }

int run_dataflow(const RunArgs &a, int dtype, int *flags) {
  switch (dtype) {
    case APSP_I32: return launch_dataflow<int32_t>(a, flags);
    case APSP_F32: return launch_dataflow<float>(a, flags);
    case APSP_I16: return launch_dataflow<int16_t>(a, flags);
  }
  return APSP_EINVAL;
}

}  // namespace apsp
