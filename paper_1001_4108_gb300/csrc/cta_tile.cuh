// One CTA working on S x S tiles of a matrix with an M x M register block
// per thread: the tile moves of the batched kernels and of the one-launch
// small-matrix solver, the min-plus tile product of phases 2 and 3 (Fig. 2)
// with operands in shared memory, and the phase-1 closure of a diagonal tile.
// Every candidate is one rounded sum and the minimum is exact, so these give
// the same values, element for element, as the stage kernels at the same S.
#pragma once

#include "apsp_common.cuh"

#ifndef APSP_BATCH64_CTAS
#define APSP_BATCH64_CTAS 3
#endif

namespace apsp {

// Kernel shape: tile side S (= k-block depth inside the CTA) and an M x M
// register block per thread, (S/M)^2 threads; rows M*ty+a, columns M*tx+c.
template <int S, int M> struct BShape {
  static constexpr int Q = S / M;                 // threads per dimension
  static constexpr int NT = Q * Q;
  static constexpr int LD = S + 4;                // padded shared-memory row stride
  // three tiles, the phase-1 row and column buffers (4 S words each), a slot
  static constexpr size_t SMEM = 3 * (size_t)S * LD * 4 + 8 * (size_t)S * 4 + 16;
  // CTAs per SM the register budget is sized for (s 64: APSP_BATCH64_CTAS,
  // which the shared memory allows; 0 = no bound)
  static constexpr int MIN_BLOCKS = S == 64 ? APSP_BATCH64_CTAS : 0;
};

// Thread -> block of a tile: each warp covers 4 block rows x 8 block columns
// (4M rows x 8M columns of the tile), so that the warps whose rows or columns
// all lie outside the matrix can skip their arithmetic as a whole (an idle
// lane inside a working warp saves nothing).  Needs (S/M) % 8 == 0.
template <int S, int M>
__device__ __forceinline__ void block_of_thread(int t, int &ty, int &tx) {
  constexpr int Q = S / M;
  static_assert(Q % 8 == 0 && (Q * Q) % 32 == 0, "whole warps of 4 x 8 blocks");
  constexpr int WC = Q / 8;  // warps across the tile
  const int w = t / 32, l = t % 32;
  ty = 4 * (w / WC) + l / 8;
  tx = 8 * (w % WC) + l % 8;
}

// Whether the warp holding block (ty, tx) has any element with row < rows
// and column < cols (uniform over the warp).
template <int M>
__device__ __forceinline__ bool warp_has_work(int ty, int tx, int rows, int cols) {
  return __any_sync(0xffffffffu, M * ty < rows && M * tx < cols);
}

// Reinterprets a 32-bit word as the compute type (int32 or fp32).
template <typename C> __device__ __forceinline__ C word_as(int v);
template <> __device__ __forceinline__ int32_t word_as<int32_t>(int v) { return v; }
template <> __device__ __forceinline__ float word_as<float>(int v) { return __int_as_float(v); }

// A global load; CG = true reads through L2 only (cp.async.cg-like: no L1
// line of another SM's earlier write can be hit).
template <bool CG, typename X>
__device__ __forceinline__ X gload(const X *p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// Global <-> register moves of one S x S tile, M x M elements per thread
// (rows M ty + a, columns M tx + c).  `vec`: 32-bit elements, 16-byte
// aligned matrix and rows (ld % 4 == 0), so that with M = 4 each row of a
// thread's block moves as one 128-bit access.  CG: loads bypass L1.
template <typename T, int S, int M, bool CG = false>
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
            const int4 v = gload<CG>(reinterpret_cast<const int4 *>(p + a * ld));
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
        for (int c = 0; c < M; ++c) x[a][c] = Arith<T>::load(gload<CG>(p + a * ld + c));
      return;
    }
#pragma unroll
    for (int a = 0; a < M; ++a)
#pragma unroll
      for (int c = 0; c < M; ++c) {
        const int64_t gi = r0 + M * ty + a, gj = c0 + M * tx + c;
        x[a][c] = (gi < n && gj < n) ? Arith<T>::load(gload<CG>(d + gi * ld + gj)) : Arith<T>::inf();
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
// sequential k steps (rounded up to M; the padding k's are infinity) on an
// M x M register block per thread (M = 2 or 4) -- stores it (clamped in the
// last stage) and leaves it in Ds (padded rows).  Ends with a barrier.
//
// Two k steps per barrier.  Before steps k and k + 1 the owners publish rows
// k, k + 1 and columns k, k + 1 as they stand after step k - 1 (a double
// buffer: rowbuf and colbuf hold 4 S values each).  Every thread then does
// step k, brings its own copies of row k + 1 and column k + 1 up to date with
// step k -- from x[k+1][k] and x[k][k+1], which step k leaves unchanged
// (x[k][k] >= 0) -- and does step k + 1.  Each of those values is computed
// from the same two operands as the owner's copy, so the tile is the same,
// bit for bit, as with one barrier per step.
template <typename T, int S, int M, bool CG = false>
__device__ __forceinline__ void close_diag(T *d, int64_t ld, int64_t n, int64_t p0, int kvalid, bool last,
                                           bool vec, typename Arith<T>::C *Ds, typename Arith<T>::C *rowbuf,
                                           typename Arith<T>::C *colbuf, int ty, int tx) {
  static_assert(M == 2 || M == 4, "pairs of k steps within one thread's rows");
  using C = typename Arith<T>::C;
  using IO = TileIO<T, S, M, CG>;
  C x[M][M];
  IO::load(d, ld, n, p0, p0, ty, tx, x, vec);
  if (ty == 0) {
#pragma unroll
    for (int c = 0; c < M; ++c) {
      rowbuf[M * tx + c] = x[0][c];
      rowbuf[S + M * tx + c] = x[1][c];
    }
  }
  if (tx == 0) {
#pragma unroll
    for (int a = 0; a < M; ++a) {
      colbuf[M * ty + a] = x[a][0];
      colbuf[S + M * ty + a] = x[a][1];
    }
  }
  // Warps whose rows or columns all lie beyond the k-block's vertices hold
  // padding only (never stored): they skip the arithmetic and keep the
  // infinity they loaded, which they still publish when they own a pivot
  // row or column -- every value that reaches a real entry is then a real
  // distance or a sum involving infinity, as without the skip.
  const bool work = warp_has_work<M>(ty, tx, kvalid, kvalid);
  for (int kq = 0; kq < (kvalid + M - 1) / M; ++kq) {
#pragma unroll
    for (int h = 0; h < M / 2; ++h) {
      const int g = kq * (M / 2) + h;  // pair of steps k0, k0 + 1
      const int k0 = 2 * g;
      __syncthreads();
      if (work) {
        const C *rb = rowbuf + (g & 1) * 2 * S;
        const C *cb = colbuf + (g & 1) * 2 * S;
        C r0[M], r1[M], c0[M], c1[M];
#pragma unroll
        for (int c = 0; c < M; ++c) {
          r0[c] = rb[M * tx + c];
          r1[c] = rb[S + M * tx + c];
        }
#pragma unroll
        for (int a = 0; a < M; ++a) {
          c0[a] = cb[M * ty + a];
          c1[a] = cb[S + M * ty + a];
        }
        const C p10 = rb[S + k0];  // x[k0+1][k0]
        const C p01 = rb[k0 + 1];  // x[k0][k0+1]
        // step k0
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
          for (int c = 0; c < M; ++c) x[a][c] = Arith<T>::relax(x[a][c], c0[a], r0[c]);
#pragma unroll
        for (int c = 0; c < M; ++c) r1[c] = Arith<T>::relax(r1[c], p10, r0[c]);
#pragma unroll
        for (int a = 0; a < M; ++a) c1[a] = Arith<T>::relax(c1[a], c0[a], p01);
        // step k0 + 1
#pragma unroll
        for (int a = 0; a < M; ++a)
#pragma unroll
          for (int c = 0; c < M; ++c) x[a][c] = Arith<T>::relax(x[a][c], c1[a], r1[c]);
      }
      // publish rows and columns k0 + 2, k0 + 3 (local rows lr, lr + 1 of
      // their owners) for the next pair
      const int k2 = k0 + 2;
      if (k2 < S) {
        const int lr = (2 * h + 2) % M;
        C *rn = rowbuf + ((g + 1) & 1) * 2 * S;
        C *cn = colbuf + ((g + 1) & 1) * 2 * S;
        if (ty == k2 / M) {
#pragma unroll
          for (int c = 0; c < M; ++c) {
            rn[M * tx + c] = x[lr][c];
            rn[S + M * tx + c] = x[lr + 1][c];
          }
        }
        if (tx == k2 / M) {
#pragma unroll
          for (int a = 0; a < M; ++a) {
            cn[M * ty + a] = x[a][lr];
            cn[S + M * ty + a] = x[a][lr + 1];
          }
        }
      }
    }
  }
  IO::store(d, ld, n, p0, p0, ty, tx, x, last, vec);
  IO::to_smem(Ds, ty, tx, x);
  __syncthreads();
}

}  // namespace apsp
