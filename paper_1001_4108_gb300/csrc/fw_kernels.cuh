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

namespace apsp {

// ------------------------------------------------------------------ phase 1
// One CTA; the s x s diagonal tile in shared memory; s barriers.
// Within step k, row k and column k of the tile do not change (d_kk >= 0), so
// the in-place update needs no second buffer.
template <typename T, int S, int NT>
__global__ void __launch_bounds__(NT) fw_phase1(T *__restrict__ d, int64_t n, int64_t ld, int b, int last) {
  using C = typename Arith<T>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C *X = reinterpret_cast<C *>(smem_raw);
  constexpr int E = S * S / NT;   // elements per thread
  constexpr int RS = NT / S;      // row stride between a thread's elements
  const int j = threadIdx.x % S;
  const int i0 = threadIdx.x / S;
  const int64_t base = (int64_t)b * S;
  const bool cj = base + j < n;

#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = i0 + RS * r;
    const bool ok = cj && base + i < n;
    X[i * S + j] = ok ? Arith<T>::load(d[(base + i) * ld + base + j]) : Arith<T>::inf();
  }
  __syncthreads();
  for (int k = 0; k < S; ++k) {
    const C xkj = X[k * S + j];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int i = i0 + RS * r;
      X[i * S + j] = Arith<T>::relax(X[i * S + j], X[i * S + k], xkj);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int i = i0 + RS * r;
    if (cj && base + i < n) {
      const C v = X[i * S + j];
      d[(base + i) * ld + base + j] = last ? Arith<T>::finish(v) : (T)v;
    }
  }
}

// ------------------------------------------------------------------ phase 2
// 2*(R-1) CTAs: the first R-1 take the row panel tiles (b, J), the rest the
// column panel tiles (I, b).  Shared memory holds the closed diagonal tile D
// and the panel tile X.
//   row panel:    x_ij <- min(x_ij, D_ik + x_kj)
//   column panel: x_ij <- min(x_ij, x_ik + D_kj)
template <typename T, int S, int NT>
__global__ void __launch_bounds__(NT) fw_phase2(T *__restrict__ d, int64_t n, int64_t ld, int b, int R, int last) {
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
      d[(r0 + i) * ld + c0 + j] = last ? Arith<T>::finish(v) : (T)v;
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
                                                         int last, int reverse) {
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
      if (gi < n && gj < n) d[gi * ld + gj] = last ? Arith<T>::finish(acc[r][c]) : (T)acc[r][c];
    }
}

// --------------------------------------------------- phase 3 (TMA-staged)
// 4-byte element types, full k-block (k0 + S <= n), 16-byte aligned rows.
//
// CTA tile S x S, (S/8)^2 threads, 8 x 8 register micro-tile per thread:
// rows ty + G*r (r < 8), columns h*S/2 + 4*tx + c (h < 2, c < 4), G = S/8.
// The two panels stream through shared memory in k-slices of 32 (the staged
// load of Sec. 4.2) filled by TMA into a 2-deep ring guarded by mbarriers:
//   A slice = column panel rows of tile I x 32 k's, 128-byte swizzled rows
//             (16-byte chunk c of row i stored at chunk c ^ (i % 8)), so the
//             8 rows a warp reads for one k-quad hit distinct banks;
//   B slice = 32 k's x S columns of tile J, plain row-major.
// The C tile goes global -> registers with 128-bit loads issued before the
// first wait, so they overlap the first TMA copies.
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

// 128-bit shared/global accesses of four consecutive 4-byte elements.
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

template <typename T, int S>
__global__ void __launch_bounds__(P3Tma<S>::TPB, P3Tma<S>::MIN_BLOCKS)
    fw_phase3_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  T *__restrict__ d, int64_t n, int64_t ld, int b, int last, int reverse, int *err) {
  using P = P3Tma<S>;
  constexpr int G = P::G;
  constexpr int KS = P::KS;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  T *As = reinterpret_cast<T *>(base);
  T *Bs = reinterpret_cast<T *>(base + P::STAGES * P::A_BYTES);
  uint64_t *full = reinterpret_cast<uint64_t *>(base + P::STAGES * (P::A_BYTES + P::B_BYTES));

  const int tid = threadIdx.x;
  const int tx = tid % G, ty = tid / G;
  const int It = skip_pivot(blockIdx.y, b), Jt = skip_pivot(blockIdx.x, b);
  const int64_t I0 = (int64_t)It * S, J0 = (int64_t)Jt * S;
  const int k0 = b * S;

  if (tid == 0) {
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmB);
#pragma unroll
    for (int s = 0; s < P::STAGES; ++s) mbar_init(&full[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
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
      const T *row = d + (I0 + ty + G * r) * ld + J0 + 4 * tx;
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
        acc[r][c] = (gi < n && gj < n) ? d[gi * ld + gj] : Arith<T>::inf();
      }
  }

  bool timed_out = false;
  for (int s = 0; s < P::NSL; ++s) {
    const int st = s % P::STAGES;
    if (!mbar_wait_bounded(&full[st], (s / P::STAGES) & 1)) timed_out = true;
    const T *A = As + st * (S * KS);
    const T *B = Bs + st * (KS * S);
    const int sw = ty & 7;  // swizzle phase of every row this thread reads
#pragma unroll
    for (int qi = 0; qi < KS / 4; ++qi) {
      const int q = reverse ? KS / 4 - 1 - qi : qi;
      T a[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r) ld4<T>(A + (ty + G * r) * KS + ((q ^ sw) << 2), a[r][0], a[r][1], a[r][2], a[r][3]);
#pragma unroll
      for (int ui = 0; ui < 4; ++ui) {
        const int u = reverse ? 3 - ui : ui;
        const T *brow = B + (4 * q + u) * S + 4 * tx;
        T bv[8];
        ld4<T>(brow, bv[0], bv[1], bv[2], bv[3]);
        ld4<T>(brow + S / 2, bv[4], bv[5], bv[6], bv[7]);
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = Arith<T>::relax(acc[r][c], a[r][u], bv[c]);
      }
    }
    // every thread is done with stage st: refill it with slice s + STAGES
    if (__syncthreads_or(timed_out)) {
      if (tid == 0) atomicCAS(err, 0, (int)kDevTimeoutTma);
      return;
    }
    if (tid == 0 && s + P::STAGES < P::NSL) {
      const int s2 = s + P::STAGES;
      mbar_arrive_expect_tx(&full[st], P::A_BYTES + P::B_BYTES);
      tma_load_2d(As + st * (S * KS), &tmA, &full[st], k0 + s2 * KS, (int)I0);
      tma_load_2d(Bs + st * (KS * S), &tmB, &full[st], (int)J0, k0 + s2 * KS);
    }
  }

  if (full_tile) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      T *row = d + (I0 + ty + G * r) * ld + J0 + 4 * tx;
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
        if (gi < n && gj < n) d[gi * ld + gj] = last ? Arith<T>::finish(acc[r][c]) : acc[r][c];
      }
  }
}

}  // namespace apsp
