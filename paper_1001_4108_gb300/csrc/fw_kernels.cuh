// Kernels of one stage (k-block) of blocked Floyd-Warshall, Sec. 3.2 / Fig. 2
// of Lund & Smith, and the host loop over the stages.
//
//   phase 1  "independent block": the diagonal tile (b,b), s sequential k steps
//            whose dependencies are all inside the tile.
//   phase 2  "singly dependent blocks": tiles (b,J) and (I,b); each depends on
//            the closed diagonal tile and on itself.
//   phase 3  "doubly dependent blocks": every other tile (I,J) takes
//            d_ij = min(d_ij, min_k d_ik + d_kj) over the k-block; its inputs
//            (the two panels) are final for the stage, so the s tasks of an
//            element may run in any order (Sec. 3.2) -- this is what lets the
//            tile live in registers (Sec. 4.1) and the panels stream through
//            shared memory in k-slices (Sec. 4.2).
//
// Vertices n..n_p-1 of the padded grid (n_p = rounds * s) are isolated
// vertices: every load outside the matrix reads "infinity", nothing outside
// the matrix is stored, so they never change a real entry.
#pragma once

#include "apsp_common.cuh"
#include "tileset.h"

#include <type_traits>

namespace apsp {

// Path bookkeeping (optional, via != nullptr): via[i][j] = the stage b whose
// k-block last strictly improved d_ij.  Each store site compares the new
// value with the one it replaces; stages run in order, so the last stage to
// write is the last improvement.  The TMA-staged kernels compile it only in
// their VIA instances, so that the distance-only kernels keep their code.
template <typename C>
__device__ __forceinline__ void note_via(int16_t *via, int64_t via_ld, int64_t i, int64_t j, C now, C before, int b) {
  if (now < before) via[i * via_ld + j] = (int16_t)b;
}

// Where a phase-3 launch reads and writes its C tiles: normally the matrix
// itself (src = dst = d).  The host entry point can point the first stage's
// reads at the caller's host matrix and the last stage's writes back to it,
// so that the matrix crosses the host link inside those two stages instead
// of in separate copies.  The panels always come from the device matrix.
template <typename T>
struct CRoute {
  const T *src;
  int64_t src_ld;
  T *dst;
  int64_t dst_ld;
};

// ------------------------------------------------------------------ phase 1
// One CTA closes the diagonal tile (b, b): s sequential k steps, each a rank-1
// update x_ij <- min(x_ij, x_ik + x_kj) of the whole tile.
// The tile lives in registers, an MR x MC block per thread ((s/MR)(s/MC)
// threads); only row k and column k travel through shared memory.  Within
// step k, row k and column k do not change (d_kk >= 0), so the owners of
// row/column k+1 publish them right after their own step-k update, into the
// other half of a double buffer: one barrier per step.
template <typename T, int S, int MR, int MC>
__device__ __forceinline__ void phase1_body(T *__restrict__ d, int64_t n, int64_t ld, int b, int last,
                                            int16_t *__restrict__ via, int64_t via_ld) {
  using C = typename Arith<T>::C;
  constexpr int QC = S / MC;  // thread columns
  constexpr int U = MR > MC ? MR : MC;  // k steps per unrolled group (MR, MC in {4, 8})
  __shared__ __align__(16) C rowbuf[2][S];
  __shared__ __align__(16) C colbuf[2][S];
  const int tx = threadIdx.x % QC, ty = threadIdx.x / QC;
  const int64_t base = (int64_t)b * S;
  C x[MR][MC];
  wait_prior_grid();
#pragma unroll
  for (int a = 0; a < MR; ++a)
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int64_t gi = base + MR * ty + a, gj = base + MC * tx + c;
      x[a][c] = (gi < n && gj < n) ? Arith<T>::load(d[gi * ld + gj]) : Arith<T>::inf();
    }
  if (ty == 0) {
#pragma unroll
    for (int c = 0; c < MC; ++c) rowbuf[0][MC * tx + c] = x[0][c];
  }
  if (tx == 0) {
#pragma unroll
    for (int a = 0; a < MR; ++a) colbuf[0][MR * ty + a] = x[a][0];
  }
  for (int kq = 0; kq < S / U; ++kq) {
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = U * kq + u;
      __syncthreads();
      C rk[MC], ck[MR];
#pragma unroll
      for (int c = 0; c < MC; ++c) rk[c] = rowbuf[k & 1][MC * tx + c];
#pragma unroll
      for (int a = 0; a < MR; ++a) ck[a] = colbuf[k & 1][MR * ty + a];
#pragma unroll
      for (int a = 0; a < MR; ++a)
#pragma unroll
        for (int c = 0; c < MC; ++c) x[a][c] = Arith<T>::relax(x[a][c], ck[a], rk[c]);
      // publish row k + 1 (local row (u + 1) % MR of thread row (k + 1) / MR)
      // and column k + 1 (local column (u + 1) % MC of thread column (k + 1) / MC)
      const int k1 = k + 1;
      if (k1 < S) {
        if (ty == k1 / MR) {
#pragma unroll
          for (int c = 0; c < MC; ++c) rowbuf[k1 & 1][MC * tx + c] = x[(u + 1) % MR][c];
        }
        if (tx == k1 / MC) {
#pragma unroll
          for (int a = 0; a < MR; ++a) colbuf[k1 & 1][MR * ty + a] = x[a][(u + 1) % MC];
        }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < MR; ++a)
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      const int64_t gi = base + MR * ty + a, gj = base + MC * tx + c;
      if (gi < n && gj < n) {
        if (via) note_via(via, via_ld, gi, gj, x[a][c], Arith<T>::load(d[gi * ld + gj]), b);
        d[gi * ld + gj] = last ? Arith<T>::finish(x[a][c]) : (T)x[a][c];
      }
    }
}

// Alone on the GPU: 4 x 4 blocks, the most threads (latency bound).
template <typename T, int S>
__global__ void __launch_bounds__((S / 4) * (S / 4)) fw_phase1(T *__restrict__ d, int64_t n, int64_t ld, int b,
                                                               int last, int16_t *via, int64_t via_ld) {
  phase1_body<T, S, 4, 4>(d, n, ld, b, last, via, via_ld);
}

// Beside phase 3 (lookahead schedule): 8 x 4 blocks and at most 64 registers
// per thread, so that the CTA fits on an SM next to a phase-3 CTA
// (S = 128: 512 threads x 64 registers = 32768).
template <typename T, int S>
__global__ void __launch_bounds__((S / 8) * (S / 4), S == 128 ? 2 : 4)
    fw_phase1_side(T *__restrict__ d, int64_t n, int64_t ld, int b, int last, int16_t *via, int64_t via_ld) {
  phase1_body<T, S, 8, 4>(d, n, ld, b, last, via, via_ld);
}

// ------------------------------------------------------------------ phase 2
// 2*(R-1) CTAs: the first R-1 take the row panel tiles (b, J), the rest the
// column panel tiles (I, b).  Shared memory holds the closed diagonal tile D
// and the panel tile X.
//   row panel:    x_ij <- min(x_ij, D_ik + x_kj)
//   column panel: x_ij <- min(x_ij, x_ik + D_kj)
//
// With bp != nullptr the row panel tiles are also stored, k-pair interleaved,
// into bp: element (k, j) of the pivot row block goes to
// bp[(k / 2) * bp_ld + 2 * j + (k % 2)] (j = global column, padding included),
// the layout the packed fp32 phase-3 kernel reads.
template <typename T, int S, int NT>
__global__ void __launch_bounds__(NT) fw_phase2(T *__restrict__ d, int64_t n, int64_t ld, int b, int R, int last,
                                                T *__restrict__ bp, int64_t bp_ld, int16_t *__restrict__ via,
                                                int64_t via_ld) {
  using C = typename Arith<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *D = reinterpret_cast<C *>(smem_raw);
  C *X = D + S * S;
  constexpr int E = S * S / NT;
  constexpr int RS = NT / S;
  const int j = threadIdx.x % S;
  const int i0 = threadIdx.x / S;
  const bool row_panel = (int)blockIdx.x < R - 1;
  const int other = skip_pivot(row_panel ? blockIdx.x : blockIdx.x - (R - 1), b);
  const int64_t pb = (int64_t)b * S;
  const int64_t r0 = row_panel ? pb : (int64_t)other * S;
  const int64_t c0 = row_panel ? (int64_t)other * S : pb;
  wait_prior_grid();

#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = i0 + RS * r;
    const bool okd = pb + i < n && pb + j < n;
    D[i * S + j] = okd ? Arith<T>::load(d[(pb + i) * ld + pb + j]) : Arith<T>::inf();
    const bool okx = r0 + i < n && c0 + j < n;
    X[i * S + j] = okx ? Arith<T>::load(d[(r0 + i) * ld + c0 + j]) : Arith<T>::inf();
  }
  __syncthreads();
  if (row_panel) {
    for (int k = 0; k < S; ++k) {
      const C xkj = X[k * S + j];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = i0 + RS * r;
        X[i * S + j] = Arith<T>::relax(X[i * S + j], D[i * S + k], xkj);
      }
      __syncthreads();
    }
  } else {
    for (int k = 0; k < S; ++k) {
      const C dkj = D[k * S + j];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        const int i = i0 + RS * r;
        X[i * S + j] = Arith<T>::relax(X[i * S + j], X[i * S + k], dkj);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = i0 + RS * r;
    if (r0 + i < n && c0 + j < n) {
      const C v = X[i * S + j];
      if (via) note_via(via, via_ld, r0 + i, c0 + j, v, Arith<T>::load(d[(r0 + i) * ld + c0 + j]), b);
      d[(r0 + i) * ld + c0 + j] = last ? Arith<T>::finish(v) : (T)v;
    }
  }
  if (bp && row_panel) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = i0 + RS * r;
      bp[(int64_t)(i >> 1) * bp_ld + 2 * (c0 + j) + (i & 1)] = (T)X[i * S + j];
    }
  }
}

// ------------------------------------------------------- phase 3 (generic)
// Any alignment, any partial k-block.  One CTA per doubly dependent tile,
// 256 threads, (S/16) x (S/16) register micro-tile per thread (Sec. 4.1);
// both panels are read once into shared memory with "infinity" outside the
// matrix.  grid = (R-1, R-1).
template <typename T, int S>
__global__ void __launch_bounds__(256) fw_phase3_generic(T *__restrict__ d, int64_t n, int64_t ld, int b,
                                                         int last, int reverse, int16_t *__restrict__ via,
                                                         int64_t via_ld) {
  using C = typename Arith<T>::C;
  constexpr int M = S / 16;
  constexpr int AS = S + 1;  // padded row stride of the column panel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *A = reinterpret_cast<C *>(smem_raw);  // [S][S+1]: rows of tile I, k-block columns
  C *B = A + S * AS;                       // [S][S]:   k-block rows, columns of tile J
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int64_t I0 = (int64_t)skip_pivot(blockIdx.y, b) * S;
  const int64_t J0 = (int64_t)skip_pivot(blockIdx.x, b) * S;
  const int64_t K0 = (int64_t)b * S;
  wait_prior_grid();

  for (int e = threadIdx.x; e < S * S; e += 256) {
    const int r = e / S, c = e % S;
    A[r * AS + c] = (I0 + r < n && K0 + c < n) ? Arith<T>::load(d[(I0 + r) * ld + K0 + c]) : Arith<T>::inf();
    B[r * S + c] = (K0 + r < n && J0 + c < n) ? Arith<T>::load(d[(K0 + r) * ld + J0 + c]) : Arith<T>::inf();
  }
  C acc[M][M];
#pragma unroll
  for (int r = 0; r < M; ++r)
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int64_t gi = I0 + ty + 16 * r, gj = J0 + tx + 16 * c;
      acc[r][c] = (gi < n && gj < n) ? Arith<T>::load(d[gi * ld + gj]) : Arith<T>::inf();
    }
  __syncthreads();
  for (int kk = 0; kk < S; ++kk) {
    const int k = reverse ? S - 1 - kk : kk;
    C a[M], bv[M];
#pragma unroll
    for (int r = 0; r < M; ++r) a[r] = A[(ty + 16 * r) * AS + k];
#pragma unroll
    for (int c = 0; c < M; ++c) bv[c] = B[k * S + tx + 16 * c];
#pragma unroll
    for (int r = 0; r < M; ++r)
#pragma unroll
      for (int c = 0; c < M; ++c) acc[r][c] = Arith<T>::relax(acc[r][c], a[r], bv[c]);
  }
#pragma unroll
  for (int r = 0; r < M; ++r)
#pragma unroll
    for (int c = 0; c < M; ++c) {
      const int64_t gi = I0 + ty + 16 * r, gj = J0 + tx + 16 * c;
      if (gi < n && gj < n) {
        if (via) note_via(via, via_ld, gi, gj, acc[r][c], Arith<T>::load(d[gi * ld + gj]), b);
        d[gi * ld + gj] = last ? Arith<T>::finish(acc[r][c]) : (T)acc[r][c];
      }
    }
}

// ------------------------------------------- phases 2 and 3 (TMA-staged)
// One kernel updates a set of S x S tiles C = (I, J) with
//     c_ij <- min(c_ij, min_{k in block b} a_ik + b_kj),
//     a = tile (I, b) of the matrix, b = tile (b, J) of the matrix,
// for 4-byte element types, a full k-block (k0 + S <= n) and 16-byte aligned
// rows.
//   phase 3 (MODE 0): doubly dependent tiles I != b, J != b, those of the
//            tile set `ts`, one per CTA.  Their operands are final for the
//            stage.
//   phase 2 (MODE 1): the singly dependent tiles; blockIdx.x < R-1 takes the
//            row panel tile (b, J), the rest the column panel tile (I, b).
//            After phase 1 the diagonal tile D is closed (its own shortest
//            paths, zero diagonal), and the k-sequential loop of Fig. 2 on a
//            row panel tile X reaches exactly min_k D_ik + X_kj: a path from
//            i to j through block b leaves the block once, at its last
//            vertex k.  So the row panel is the min-plus product D (x) X and
//            the column panel X (x) D, both of the form above, with a = D or
//            b = D.  A CTA reads its own tile as an operand; all its TMA
//            reads complete before its single store at the end.
//            (Integers: exactly the sequential result; fp32: the same
//            shortest-path value up to the association of the additions.)
//
// CTA tile S x S, (S/8)^2 threads, 8 x 8 register micro-tile per thread:
// rows ty + G*r (r < 8), columns h*S/2 + 4*tx + c (h < 2, c < 4), G = S/8.
// The operands stream through shared memory in k-slices of 32 (the staged
// load of Sec. 4.2), filled by TMA into a 2-deep ring guarded by mbarriers:
//   A slice = rows of tile I x 32 k's, 128-byte swizzled rows (16-byte chunk
//             c of row i stored at chunk c ^ (i % 8)), so the 8 rows a warp
//             reads for one k-quad hit distinct banks;
//   B slice = 32 k's x S columns of tile J, plain row-major.
// The C tile goes global -> registers with 128-bit loads issued before the
// first wait, so they overlap the first TMA copies.
//
// With bp != nullptr (phase 2, fp32) the row panel tiles are also written,
// k-pair interleaved, to bp: element (k, j) of the pivot row block goes to
// bp[(k / 2) * bp_ld + 2 * j + (k % 2)] (j = global column, padding
// included), the layout the packed fp32 phase-3 kernel reads.
template <int S> struct P3Tma {
  static constexpr int G = S / 8;
  static constexpr int TPB = G * G;
  static constexpr int KS = 32;
  static constexpr int NSL = S / KS;
  static constexpr int STAGES = 2;
  static constexpr int A_BYTES = S * KS * 4;
  static constexpr int B_BYTES = KS * S * 4;
  static constexpr int SMEM = STAGES * (A_BYTES + B_BYTES) + 1024 + 64;
  static constexpr int MIN_BLOCKS = S == 128 ? 2 : 6;
};

template <typename T>
__device__ __forceinline__ void ld4(const T *p, T &x0, T &x1, T &x2, T &x3);
template <>
__device__ __forceinline__ void ld4<int32_t>(const int32_t *p, int32_t &x0, int32_t &x1, int32_t &x2, int32_t &x3) {
  const int4 v = *reinterpret_cast<const int4 *>(p);
  x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
}
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float &x0, float &x1, float &x2, float &x3) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  x0 = v.x; x1 = v.y; x2 = v.z; x3 = v.w;
}
template <typename T>
__device__ __forceinline__ void st4(T *p, T x0, T x1, T x2, T x3);
template <>
__device__ __forceinline__ void st4<int32_t>(int32_t *p, int32_t x0, int32_t x1, int32_t x2, int32_t x3) {
  *reinterpret_cast<int4 *>(p) = make_int4(x0, x1, x2, x3);
}
template <>
__device__ __forceinline__ void st4<float>(float *p, float x0, float x1, float x2, float x3) {
  *reinterpret_cast<float4 *>(p) = make_float4(x0, x1, x2, x3);
}
// Shared-memory loads the compiler may not merge or hoist across the k-pair
// loop (keeps the 64 accumulators within two CTAs per SM worth of registers).
template <typename T>
__device__ __forceinline__ void lds2(const T *p, T &x0, T &x1) {
  uint32_t a, b;
  asm volatile("ld.shared.v2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(smem_u32(p)));
  x0 = *reinterpret_cast<T *>(&a);
  x1 = *reinterpret_cast<T *>(&b);
}
template <typename T>
__device__ __forceinline__ void lds4(const T *p, T &x0, T &x1, T &x2, T &x3) {
  uint32_t a, b, c, e;
  asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(a), "=r"(b), "=r"(c), "=r"(e) : "r"(smem_u32(p)));
  x0 = *reinterpret_cast<T *>(&a);
  x1 = *reinterpret_cast<T *>(&b);
  x2 = *reinterpret_cast<T *>(&c);
  x3 = *reinterpret_cast<T *>(&e);
}

template <typename T, int S, int MODE, bool VIA = false>
__global__ void __launch_bounds__(P3Tma<S>::TPB, P3Tma<S>::MIN_BLOCKS)
    fw_tile_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const CRoute<T> cr, int64_t n, int b, int R, const TileSet ts, int last, int reverse,
                T *__restrict__ bp, int64_t bp_ld, int16_t *__restrict__ via, int64_t via_ld, int *err) {
  using P = P3Tma<S>;
  constexpr int G = P::G;
  constexpr int KS = P::KS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  T *As = reinterpret_cast<T *>(base);
  T *Bs = reinterpret_cast<T *>(base + P::STAGES * P::A_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + P::STAGES * (P::A_BYTES + P::B_BYTES));

  int *tile_ij = reinterpret_cast<int *>(full + P::STAGES);  // (It, Jt), reread after the main loop
  RingCtl<P::STAGES> *ring = reinterpret_cast<RingCtl<P::STAGES> *>(tile_ij + 2);

  const int tid = threadIdx.x;
  const int tx = tid % G, ty = tid / G;
  int It, Jt;
  if (MODE == 0) {
    ts.tile(blockIdx.x, It, Jt);
  } else {
    const bool rp = (int)blockIdx.x < R - 1;
    It = rp ? b : skip_pivot(blockIdx.x - (R - 1), b);
    Jt = rp ? skip_pivot(blockIdx.x, b) : b;
  }
  int64_t I0 = (int64_t)It * S, J0 = (int64_t)Jt * S;
  const int k0 = b * S;

  if (tid == 0) {
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmB);
#pragma unroll
    for (int s = 0; s < P::STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    ring_ctl_init(ring, P::STAGES < P::NSL ? P::STAGES : P::NSL);
    tile_ij[0] = It;
    tile_ij[1] = Jt;
  }
  __syncthreads();
  wait_prior_grid();
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < P::STAGES && s < P::NSL; ++s) {
      mbar_arrive_expect_tx(&full[s], P::A_BYTES + P::B_BYTES);
      tma_load_2d(As + s * (S * KS), &tmA, &full[s], k0 + s * KS, (int)I0);
      tma_load_2d(Bs + s * (KS * S), &tmB, &full[s], (int)J0, k0 + s * KS);
    }
  }

  // C tile -> registers.
  const bool full_tile = I0 + S <= n && J0 + S <= n;
  T acc[8][8];
  if (full_tile) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const T *row = cr.src + (I0 + ty + G * r) * cr.src_ld + J0 + 4 * tx;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        ld4<T>(row + h * (S / 2), acc[r][4 * h], acc[r][4 * h + 1], acc[r][4 * h + 2], acc[r][4 * h + 3]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t gi = I0 + ty + G * r, gj = J0 + (c / 4) * (S / 2) + 4 * tx + (c % 4);
        acc[r][c] = (gi < n && gj < n) ? cr.src[gi * cr.src_ld + gj] : Arith<T>::inf();
      }
  }

  bool timed_out = false;
  const int sw = ty & 7;  // swizzle phase of every row this thread reads
  for (int s = 0; s < P::NSL; ++s) {
    const int st = s % P::STAGES;
    if (!timed_out && !mbar_wait_bounded(&full[st], (s / P::STAGES) & 1)) timed_out = true;
    const T *A = As + st * (S * KS) + ty * KS;
    const T *B = Bs + st * (KS * S) + 4 * tx;
    if constexpr (std::is_same<T, float>::value) {
      // fp32 (fadd + fmin, 2 issue slots per relaxation): one k-pair per
      // iteration, operands loaded per iteration, to stay spill-free.
#pragma unroll 1
      for (int pi = 0; pi < KS / 2; ++pi) {
        const int p = reverse ? KS / 2 - 1 - pi : pi;  // k-pair (2p, 2p + 1) of the slice
        const int aoff = (((p >> 1) ^ sw) << 2) + ((p & 1) << 1);
        T a[8][2];
#pragma unroll
        for (int r = 0; r < 8; ++r) lds2<T>(A + G * r * KS + aoff, a[r][0], a[r][1]);
#pragma unroll
        for (int ui = 0; ui < 2; ++ui) {
          const int u = reverse ? 1 - ui : ui;
          const T *brow = B + (2 * p + u) * S;
          T bv[8];
          lds4<T>(brow, bv[0], bv[1], bv[2], bv[3]);
          lds4<T>(brow + S / 2, bv[4], bv[5], bv[6], bv[7]);
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = Arith<T>::relax(acc[r][c], a[r][u], bv[c]);
        }
      }
    } else {
      // int32 (one DPX add-min per relaxation on the half-rate pipe): the
      // fully unrolled slice lets the compiler run the shared loads far
      // ahead of their use; issue slots are not the limit here.
#pragma unroll
      for (int qi = 0; qi < KS / 4; ++qi) {
        const int q = reverse ? KS / 4 - 1 - qi : qi;
        T a[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r) ld4<T>(A + G * r * KS + ((q ^ sw) << 2), a[r][0], a[r][1], a[r][2], a[r][3]);
#pragma unroll
        for (int ui = 0; ui < 4; ++ui) {
          const int u = reverse ? 3 - ui : ui;
          const T *brow = B + (4 * q + u) * S;
          T bv[8];
          ld4<T>(brow, bv[0], bv[1], bv[2], bv[3]);
          ld4<T>(brow + S / 2, bv[4], bv[5], bv[6], bv[7]);
#pragma unroll
          for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[r][c] = Arith<T>::relax(acc[r][c], a[r][u], bv[c]);
        }
      }
    }
    // the last warp done with stage st refills it with slice s + STAGES (no
    // CTA barrier per slice)
    if (s + P::STAGES < P::NSL)
      ring_release<P::STAGES, P::TPB / 32>(ring, st, timed_out, [&] {
        const int s2 = s + P::STAGES;
        mbar_arrive_expect_tx(&full[st], P::A_BYTES + P::B_BYTES);
        tma_load_2d(As + st * (S * KS), &tmA, &full[st], k0 + s2 * KS, lds_volatile(tile_ij) * S);
        tma_load_2d(Bs + st * (KS * S), &tmB, &full[st], lds_volatile(tile_ij + 1) * S, k0 + s2 * KS);
      });
  }
  // no CTA barrier at the end: each warp has consumed every slice it needs;
  // a warp whose wait gave up drains what may still be in flight and leaves
  if (__any_sync(0xffffffffu, timed_out)) {
    if ((tid & 31) == 0) ring_drain(ring, full, err);
    return;
  }

  // tile coordinates from shared memory: nothing of them stays live in
  // registers across the main loop
  It = lds_volatile(tile_ij);
  Jt = lds_volatile(tile_ij + 1);
  I0 = (int64_t)It * S;
  J0 = (int64_t)Jt * S;
  const bool row_panel = MODE == 1 && It == b;
  if (VIA && via) {  // path bookkeeping: compare with the values about to be replaced
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t gi = I0 + ty + G * r, gj = J0 + (c / 4) * (S / 2) + 4 * tx + (c % 4);
        if (gi < n && gj < n) note_via(via, via_ld, gi, gj, acc[r][c], cr.src[gi * cr.src_ld + gj], b);
      }
  }
  if (I0 + S <= n && J0 + S <= n) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      T *row = cr.dst + (I0 + ty + G * r) * cr.dst_ld + J0 + 4 * tx;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        T v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = last ? Arith<T>::finish(acc[r][4 * h + c]) : acc[r][4 * h + c];
        st4<T>(row + h * (S / 2), v[0], v[1], v[2], v[3]);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t gi = I0 + ty + G * r, gj = J0 + (c / 4) * (S / 2) + 4 * tx + (c % 4);
        if (gi < n && gj < n) cr.dst[gi * cr.dst_ld + gj] = last ? Arith<T>::finish(acc[r][c]) : acc[r][c];
      }
  }
  if (MODE == 1 && bp && row_panel) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int i = ty + G * r;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int64_t j = J0 + (c / 4) * (S / 2) + 4 * tx + (c % 4);
        bp[(int64_t)(i >> 1) * bp_ld + 2 * j + (i & 1)] = acc[r][c];
      }
    }
  }
}

// ------------------------------------------- phase 3, fp32 packed form
// Same tiling and TMA ring as fw_tile_tma, but two k's are consumed per
// instruction pair: a packed add.f32x2 forms (a_ik + b_kj, a_ik' + b_k'j)
// for k' = k + 1 and a three-input min folds both into the accumulator,
// i.e. acc <- min(acc, a_ik + b_kj, a_ik' + b_k'j).  Each addition is rounded
// once and the minimum is exact, so the result is bit-identical to the
// one-k-at-a-time form.
// The B operand comes from the k-pair interleaved copy of the row panel
// written by phase 2 (slice = 16 k-pairs x 2S floats), so that one 128-bit
// load yields the (k, k+1) pairs of two adjacent columns.  Thread columns:
// j = 2 (tx + G m) + e, m < 4, e < 2.
//
// blockIdx.x numbers the tiles of the launch's tile set.  FULL = true: every
// row and column of every tile is inside the matrix (interior tiles); FULL =
// false: masked loads/stores (the edge tiles of a ragged matrix).
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// (a.x + b.x, a.y + b.y), each rounded to nearest: one packed add.f32x2.
__device__ __forceinline__ float2 add2f(float2 a, float2 b) { return __fadd2_rn(a, b); }

template <int S, bool REVERSE, bool FULL, bool VIA = false>
__global__ void __launch_bounds__(P3Tma<S>::TPB, P3Tma<S>::MIN_BLOCKS)
    fw_phase3_f32x2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBp,
                    const CRoute<float> cr, int64_t n, int b, const TileSet ts, int16_t *__restrict__ via,
                    int64_t via_ld, int *err) {
  using P = P3Tma<S>;
  constexpr int G = P::G;
  constexpr int KS = P::KS;
  constexpr int KP = KS / 2;  // k-pairs per slice
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float *As = reinterpret_cast<float *>(base);
  float *Bs = reinterpret_cast<float *>(base + P::STAGES * P::A_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + P::STAGES * (P::A_BYTES + P::B_BYTES));
  RingCtl<P::STAGES> *ring = reinterpret_cast<RingCtl<P::STAGES> *>(full + P::STAGES);

  const int tid = threadIdx.x;
  const int tx = tid % G, ty = tid / G;
  int It, Jt;
  ts.tile(blockIdx.x, It, Jt);
  const int k0 = b * S;

  if (tid == 0) {
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmBp);
#pragma unroll
    for (int s = 0; s < P::STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
    ring_ctl_init(ring, P::STAGES < P::NSL ? P::STAGES : P::NSL);
  }
  __syncthreads();
  wait_prior_grid();
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < P::STAGES && s < P::NSL; ++s) {
      mbar_arrive_expect_tx(&full[s], P::A_BYTES + P::B_BYTES);
      tma_load_2d(As + s * (S * KS), &tmA, &full[s], k0 + s * KS, It * S);
      tma_load_2d(Bs + s * (KS * S), &tmBp, &full[s], 2 * Jt * S, s * KP);
    }
  }

  // C tile -> registers.  The addresses are derived from (It, Jt, ty, tx)
  // here and again after the main loop from copies the compiler cannot see
  // through, so that no address is kept live across the loop.
  float acc[8][8];
  uint64_t cbase =
      reinterpret_cast<uint64_t>(cr.src + ((int64_t)It * S + ty) * cr.src_ld + (int64_t)Jt * S + 2 * tx);
  int64_t rstride = (int64_t)G * cr.src_ld * (int64_t)sizeof(float);
  int rows_left = 0, cols_left = 0;  // (masked form) rows/cols of the tile inside the matrix, from this thread
  if (!FULL) {
    rows_left = (int)(n - ((int64_t)It * S + ty));
    cols_left = (int)(n - ((int64_t)Jt * S + 2 * tx));
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float *pc = reinterpret_cast<const float *>(cbase + r * rstride + 8 * G * m);
      if (FULL) {
        const float2 v = *reinterpret_cast<const float2 *>(pc);
        acc[r][2 * m] = v.x;
        acc[r][2 * m + 1] = v.y;
      } else {
        const bool rok = G * r < rows_left;
        acc[r][2 * m] = (rok && 2 * G * m < cols_left) ? pc[0] : Arith<float>::inf();
        acc[r][2 * m + 1] = (rok && 2 * G * m + 1 < cols_left) ? pc[1] : Arith<float>::inf();
      }
    }

  bool timed_out = false;
  const int sw = ty & 7;
  for (int s = 0; s < P::NSL; ++s) {
    const int st = s % P::STAGES;
    if (!timed_out && !mbar_wait_bounded(&full[st], (s / P::STAGES) & 1)) timed_out = true;
    const float *A = As + st * (S * KS) + ty * KS;
    const float *B = Bs + st * (KS * S) + 4 * tx;
    // One k-pair per iteration, unrolled by 2: the operands are loaded with
    // volatile shared loads, so nothing is hoisted across iterations, and the
    // unrolled pair saves the loop's own instructions on this issue-bound
    // kernel (2.9 % faster than rolled at n = 16384; by 4 or 8: 0.5 % slower
    // than by 2).
#pragma unroll 2
    for (int pi = 0; pi < KP; ++pi) {
      const int p = REVERSE ? KP - 1 - pi : pi;
      const int aoff = (((p >> 1) ^ sw) << 2) + ((p & 1) << 1);  // swizzled (k, k+1) of a row
      float2 ap[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                     : "=f"(ap[r].x), "=f"(ap[r].y)
                     : "r"(smem_u32(A + G * r * KS + aoff)));
      float4 bq[4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(bq[m].x), "=f"(bq[m].y), "=f"(bq[m].z), "=f"(bq[m].w)
                     : "r"(smem_u32(B + p * (2 * S) + 4 * G * m)));
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const float2 s0 = add2f(ap[r], make_float2(bq[m].x, bq[m].y));
          const float2 s1 = add2f(ap[r], make_float2(bq[m].z, bq[m].w));
          acc[r][2 * m] = min3f(acc[r][2 * m], s0.x, s0.y);
          acc[r][2 * m + 1] = min3f(acc[r][2 * m + 1], s1.x, s1.y);
        }
    }
    // the last warp done with stage st refills it with slice s + STAGES (no
    // CTA barrier per slice, none at the end: 1.2 % faster than a barrier
    // per slice at n = 16384)
    if (s + P::STAGES < P::NSL)
      ring_release<P::STAGES, P::TPB / 32>(ring, st, timed_out, [&] {
        const int s2 = s + P::STAGES;
        mbar_arrive_expect_tx(&full[st], P::A_BYTES + P::B_BYTES);
        tma_load_2d(As + st * (S * KS), &tmA, &full[st], k0 + s2 * KS, It * S);
        tma_load_2d(Bs + st * (KS * S), &tmBp, &full[st], 2 * Jt * S, s2 * KP);
      });
  }
  // each warp has consumed every slice it needs; one whose wait gave up
  // drains what may still be in flight and leaves
  if (__any_sync(0xffffffffu, timed_out)) {
    if ((tid & 31) == 0) ring_drain(ring, full, err);
    return;
  }

  int It2 = It, Jt2 = Jt, ty2 = ty, tx2 = tx;
  asm volatile("" : "+r"(It2), "+r"(Jt2), "+r"(ty2), "+r"(tx2));
  cbase = reinterpret_cast<uint64_t>(cr.dst + ((int64_t)It2 * S + ty2) * cr.dst_ld + (int64_t)Jt2 * S + 2 * tx2);
  rstride = (int64_t)G * cr.dst_ld * (int64_t)sizeof(float);
  if (!FULL) {
    rows_left = (int)(n - ((int64_t)It2 * S + ty2));
    cols_left = (int)(n - ((int64_t)Jt2 * S + 2 * tx2));
  }
  if (VIA && via) {  // path bookkeeping: compare with the values about to be replaced
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int64_t gi = (int64_t)It2 * S + ty2 + G * r, gj = (int64_t)Jt2 * S + 2 * tx2 + 2 * G * m + e;
          if (gi < n && gj < n) note_via(via, via_ld, gi, gj, acc[r][2 * m + e], cr.src[gi * cr.src_ld + gj], b);
        }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      float *pc = reinterpret_cast<float *>(cbase + r * rstride + 8 * G * m);
      if (FULL) {
        *reinterpret_cast<float2 *>(pc) = make_float2(acc[r][2 * m], acc[r][2 * m + 1]);
      } else {
        const bool rok = G * r < rows_left;
        if (rok && 2 * G * m < cols_left) pc[0] = acc[r][2 * m];
        if (rok && 2 * G * m + 1 < cols_left) pc[1] = acc[r][2 * m + 1];
      }
    }
}

// ------------------------------------------- strips (latency-bound launches)
// With s = 64 the panel launch of a stage has 2(R-1) tiles and the cross
// launch of the lookahead schedule about as many; for small n that is fewer
// tiles than SMs, and each runs as one 64-thread CTA on the stage's critical
// path.  Here every tile is cut into four strips, one CTA each, so that four
// times as many SMs share the work: 64 x 16 column strips, and 16 x 64 row
// strips for the column-panel tiles (I, b).  The cut follows what each
// output reads:
//   row panel (b, J)     x_ij <- min(x_ij, min_k D_ik + x_kj): column j only;
//   column panel (I, b)  x_ij <- min(x_ij, min_k x_ik + D_kj): row i only;
//   other tiles          the two panels only;
// so no strip reads what another strip of the launch writes.  D is closed
// with a zero diagonal, so taking x_kj (x_ik) from before the update gives
// the closure of the singly dependent tile: for integers the values of the
// sequential k loop, and for fp32 those of the TMA kernels (every candidate is
// one rounded sum and min is exact), so the result does not depend on which
// kernel ran.  Needs a full k-block and 16-byte aligned rows (ld % 4 == 0),
// as the TMA kernels do.
//
// Thread (tr, tc) of a RS x CS strip owns rows 4tr..4tr+3 and columns
// 4tc..4tc+3; per k it reads four A values (shared memory keeps A transposed,
// AT[k][r]) and four B values, each as one 128-bit load.
template <typename T>
struct Vec4;
template <> struct Vec4<float> { using V = float4; };
template <> struct Vec4<int32_t> { using V = int4; };

// Elements j..j+3 of a row (j % 4 == 0), "infinity" from column n on; columns
// n..ld-1 are not read.
template <typename T>
__device__ __forceinline__ typename Vec4<T>::V load_row4(const T *row, int64_t j, int64_t n) {
  using V = typename Vec4<T>::V;
  const T inf = Arith<T>::inf();
  if (j + 4 <= n) return *reinterpret_cast<const V *>(row + j);
  return V{j < n ? row[j] : inf, j + 1 < n ? row[j + 1] : inf, j + 2 < n ? row[j + 2] : inf, inf};
}

template <typename T, int S, int RS, int CS, bool VIA>
__device__ __forceinline__ void strip_body(const CRoute<T> &cr, const T *__restrict__ d, int64_t n, int64_t ld, int b,
                                           int64_t I0, int64_t J0, int last, int reverse, T *__restrict__ bp,
                                           int64_t bp_ld, int16_t *__restrict__ via, int64_t via_ld, T *sm) {
  using V = typename Vec4<T>::V;
  T *AT = sm;            // [S][RS]
  T *Bs = sm + S * RS;   // [S][CS]
  constexpr int TC = CS / 4;
  static_assert((RS / 4) * TC == 64, "64 threads, 4 x 4 each");
  const int tid = threadIdx.x;
  const int tr = tid / TC, tc = tid % TC;
  const int64_t K0 = (int64_t)b * S;
  const T inf = Arith<T>::inf();

  // All global loads are issued before the first shared-memory store, so
  // that their latencies overlap.
  // A (rows I0.., the k-block's columns) -> AT[k][r]: the thread index runs
  // along r, so the transposing stores hit consecutive banks.
  constexpr int NA = RS * (S / 4) / 64, NB = S * (CS / 4) / 64;
  V av[NA], bv[NB];
#pragma unroll
  for (int u = 0; u < NA; ++u) {
    const int e = tid + 64 * u, r = e % RS, c4 = e / RS;
    av[u] = I0 + r < n ? *reinterpret_cast<const V *>(d + (I0 + r) * ld + K0 + 4 * c4) : V{inf, inf, inf, inf};
  }
  // B (the k-block's rows, columns J0..) -> Bs[k][c]
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int e = tid + 64 * u, k = e / (CS / 4), c4 = e % (CS / 4);
    bv[u] = load_row4(d + (K0 + k) * ld, J0 + 4 * c4, n);
  }
  // C -> registers
  const int64_t gi0 = I0 + 4 * tr, gj0 = J0 + 4 * tc;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const V v = gi0 + a < n ? load_row4(cr.src + (gi0 + a) * cr.src_ld, gj0, n) : V{inf, inf, inf, inf};
    acc[a][0] = v.x; acc[a][1] = v.y; acc[a][2] = v.z; acc[a][3] = v.w;
  }
#pragma unroll
  for (int u = 0; u < NA; ++u) {
    const int e = tid + 64 * u, r = e % RS, c4 = e / RS;
    AT[(4 * c4 + 0) * RS + r] = av[u].x;
    AT[(4 * c4 + 1) * RS + r] = av[u].y;
    AT[(4 * c4 + 2) * RS + r] = av[u].z;
    AT[(4 * c4 + 3) * RS + r] = av[u].w;
  }
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int e = tid + 64 * u, k = e / (CS / 4), c4 = e % (CS / 4);
    *reinterpret_cast<V *>(Bs + k * CS + 4 * c4) = bv[u];
  }
  __syncthreads();
#pragma unroll 8
  for (int kk = 0; kk < S; ++kk) {
    const int k = reverse ? S - 1 - kk : kk;
    const V ak = *reinterpret_cast<const V *>(AT + k * RS + 4 * tr);
    const V bk = *reinterpret_cast<const V *>(Bs + k * CS + 4 * tc);
    const T ar[4] = {ak.x, ak.y, ak.z, ak.w};
    const T br[4] = {bk.x, bk.y, bk.z, bk.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[a][c] = Arith<T>::relax(acc[a][c], ar[a], br[c]);
  }
  // the row panel also goes to the k-pair interleaved workspace (padding
  // columns included) for the packed fp32 phase 3
  if (bp) {
#pragma unroll
    for (int a = 0; a < 4; a += 2)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int i = 4 * tr + a;  // k within the block
        T *p = bp + (int64_t)(i >> 1) * bp_ld + 2 * (gj0 + c);
        p[0] = acc[a][c];
        p[1] = acc[a + 1][c];
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t gi = gi0 + a;
    if (gi >= n) continue;
    if (VIA) {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (gj0 + c < n) note_via(via, via_ld, gi, gj0 + c, acc[a][c], cr.src[gi * cr.src_ld + gj0 + c], b);
    }
    T o[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) o[c] = last ? Arith<T>::finish(acc[a][c]) : acc[a][c];
    if (gj0 + 4 <= n) {
      *reinterpret_cast<V *>(cr.dst + gi * cr.dst_ld + gj0) = V{o[0], o[1], o[2], o[3]};
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c)
        if (gj0 + c < n) cr.dst[gi * cr.dst_ld + gj0 + c] = o[c];
    }
  }
}

// MODE 0: the tiles of `ts` (phase 3, C read and written through cr);
// MODE 1: the 2(R-1) panel tiles of stage b (phase 2, C in the matrix).
// Four CTAs per tile; bp (MODE 1 only) receives the row panel.
template <typename T, int S, int MODE, bool VIA = false>
__global__ void __launch_bounds__(64) fw_strip(const CRoute<T> cr, const T *__restrict__ d, int64_t n, int64_t ld,
                                               int b, int R, const TileSet ts, int last, int reverse,
                                               T *__restrict__ bp, int64_t bp_ld, int16_t *__restrict__ via,
                                               int64_t via_ld) {
  static_assert(S == 64, "strips are cut from 64 x 64 tiles");
  __shared__ __align__(16) T sm[S * (S + S / 4)];  // A and B of one strip
  const int t = blockIdx.x / 4, q = blockIdx.x % 4;
  int It, Jt;
  if (MODE == 0) {
    ts.tile(t, It, Jt);
  } else {
    const bool rp = t < R - 1;
    It = rp ? b : skip_pivot(t - (R - 1), b);
    Jt = rp ? skip_pivot(t, b) : b;
  }
  wait_prior_grid();
  const int64_t I0 = (int64_t)It * S, J0 = (int64_t)Jt * S;
  if (MODE == 1 && Jt == b)  // column panel: row strips
    strip_body<T, S, S / 4, S, VIA>(cr, d, n, ld, b, I0 + q * (S / 4), J0, last, reverse, nullptr, 0, via, via_ld,
                                    sm);
  else
    strip_body<T, S, S, S / 4, VIA>(cr, d, n, ld, b, I0, J0 + q * (S / 4), last, reverse,
                                    MODE == 1 ? bp : nullptr, bp_ld, via, via_ld, sm);
}

}  // namespace apsp
