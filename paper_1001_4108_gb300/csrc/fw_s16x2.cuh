// Phases 2 and 3 of a stage (Sec. 3.2 / Fig. 2) on int16 matrices, two
// columns per 32-bit lane (DPX viaddmin.s16x2).  Kept apart from the fp32 and
// int32 stage kernels of fw_kernels.cuh, whose helpers it uses.
#pragma once

#include "fw_kernels.cuh"

namespace apsp {

// --------------------------------------- phases 2 and 3, packed int16x2
// int16 matrices (weights >= 0, (n-1) Wmax < 16383): two adjacent columns
// are relaxed per 32-bit lane with one DPX viaddmin.s16x2:
//     (c_ij, c_ij') <- min((a_ik, a_ik) + (b_kj, b_kj'), (c_ij, c_ij')),
// each half an exact 16-bit add-min (sums <= 32766, no wrap-around).
// CTA tile S x S elements = S rows x S/2 column pairs; (S/8)^2 threads;
// per thread 8 rows (ty + G*r) x 4 column pairs (4*tx .. 4*tx+3, i.e. 8
// consecutive int16 columns): 32 packed accumulators.
//   MODE 0 (phase 3, tiles I != b, J != b): A = the column panel as
//          replicated words (a | a << 16) from the workspace, written by
//          phase 2 (rows of the whole matrix x S k's, 128-byte swizzled).
//   MODE 1 (phase 2, row and column panel tiles, as for fw_tile_tma): A comes
//          from the int16 matrix and each k is replicated in registers with a
//          byte permute; column panel CTAs write their updated tile, as
//          replicated words, into the workspace for phase 3.
// B = k-slices of tile (b, J) of the int16 matrix (32 k's x S/2 pairs).
template <int S> struct P3S16 {
  static constexpr int G = S / 8;
  static constexpr int TPB = G * G;
  static constexpr int KS = 32;
  static constexpr int NSL = S / KS;
  static constexpr int STAGES = 2;
  static constexpr int A_BYTES_REP = S * KS * 4;  // MODE 0
  static constexpr int A_BYTES_16 = S * KS * 2;   // MODE 1
  static constexpr int B_BYTES = KS * S * 2;
  // Phase 3 at s = 128 also stages the C tile in shared memory (below).
  static constexpr bool C_SMEM = S == 128;
  static constexpr int C_BYTES = C_SMEM ? S * S * 2 : 0;
  static constexpr int SMEM = STAGES * (A_BYTES_REP + B_BYTES) + 1024 + 64;
  static constexpr int SMEM_P3 = SMEM + C_BYTES;
};

__device__ __forceinline__ uint32_t rep_lo(uint32_t w) { return __byte_perm(w, 0, 0x1010); }
__device__ __forceinline__ uint32_t rep_hi(uint32_t w) { return __byte_perm(w, 0, 0x3232); }

//
// Deferred C (phase 3, s = 128): the accumulators start at "infinity" and the
// k-block runs right away; the C tile travels by TMA into shared memory
// meanwhile and is folded in at the end, c <- min(c, min_k a_ik + b_kj).  The
// minimum is exact and every value is <= 16383, so this equals starting from
// c.  In the plain form every CTA of a wave first waits for its C tile, and
// the CTAs of a wave, all equally long, issue those loads together.
template <int S, int MODE, bool VIA = false>
__global__ void __launch_bounds__(P3S16<S>::TPB, S == 128 ? 2 : 8)
    fw_tile_s16x2(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmC, int16_t *__restrict__ d, int64_t n, int64_t ld, int b,
                  int R, const TileSet ts, int reverse, uint32_t *__restrict__ arep, int16_t *__restrict__ via,
                  int64_t via_ld, int *err) {
  using P = P3S16<S>;
  constexpr int G = P::G;
  constexpr int KS = P::KS;
  constexpr int A_BYTES = MODE == 0 ? P::A_BYTES_REP : P::A_BYTES_16;
  constexpr bool DEFER_C = MODE == 0 && P::C_SMEM;
  constexpr int C_BYTES = DEFER_C ? P::C_BYTES : 0;
  extern __shared__ unsigned char smem_raw[];
  unsigned char *base =
      reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char *As = base;
  unsigned char *Bs = base + P::STAGES * A_BYTES;
  unsigned char *Cs = Bs + P::STAGES * P::B_BYTES;  // C tile, S rows x S int16 (deferred form)
  uint64_t *full = reinterpret_cast<uint64_t *>(Cs + C_BYTES);
  uint64_t *cbar = full + P::STAGES;

  int *tile_ij = reinterpret_cast<int *>(cbar + 1);  // (It, Jt), reread after the main loop
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
    if (DEFER_C) mbar_init(cbar, 1);
    fence_mbar_init();
    ring_ctl_init(ring, P::STAGES < P::NSL ? P::STAGES : P::NSL);
    tile_ij[0] = It;
    tile_ij[1] = Jt;
  }
  __syncthreads();
  wait_prior_grid();
  auto issue = [&](int s, int st) {
    const int i0 = lds_volatile(tile_ij) * S, j0 = lds_volatile(tile_ij + 1) * S;
    mbar_arrive_expect_tx(&full[st], A_BYTES + P::B_BYTES);
    if (MODE == 0)
      tma_load_2d(As + st * A_BYTES, &tmA, &full[st], s * KS, i0);  // workspace: x = k within block
    else
      tma_load_2d(As + st * A_BYTES, &tmA, &full[st], k0 + s * KS, i0);
    tma_load_2d(Bs + st * P::B_BYTES, &tmB, &full[st], j0, k0 + s * KS);
  };
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < P::STAGES && s < P::NSL; ++s) issue(s, s);
  }
  // the C tile after the first slices: it is needed only at the end, and
  // issued first it delays them (measured: about 0.5-1 % on the launch)
  if (DEFER_C && tid == 0) {
    mbar_arrive_expect_tx(cbar, P::C_BYTES);
    tma_load_2d(Cs, &tmC, cbar, Jt * S, It * S);
  }

  // C tile -> registers: 8 rows x 4 column pairs (deferred form: infinity).
  const bool full_tile = I0 + S <= n && J0 + S <= n;
  uint32_t acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t gi = I0 + ty + G * r;
    const int64_t gj = J0 + 8 * tx;
    if (DEFER_C) {
#pragma unroll
      for (int m = 0; m < 4; ++m) acc[r][m] = 16383u | (16383u << 16);
    } else if (full_tile) {
      const uint4 v = *reinterpret_cast<const uint4 *>(d + gi * ld + gj);
      acc[r][0] = v.x; acc[r][1] = v.y; acc[r][2] = v.z; acc[r][3] = v.w;
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const uint32_t lo = (gi < n && gj + 2 * m < n) ? (uint16_t)d[gi * ld + gj + 2 * m] : 16383u;
        const uint32_t hi = (gi < n && gj + 2 * m + 1 < n) ? (uint16_t)d[gi * ld + gj + 2 * m + 1] : 16383u;
        acc[r][m] = lo | (hi << 16);
      }
    }
  }

  bool timed_out = false;
  for (int s = 0; s < P::NSL; ++s) {
    const int st = s % P::STAGES;
    if (!timed_out && !mbar_wait_bounded(&full[st], (s / P::STAGES) & 1)) timed_out = true;
    const uint32_t *Bw = reinterpret_cast<const uint32_t *>(Bs + st * P::B_BYTES) + 4 * tx;  // row: S/2 words
#pragma unroll
    for (int qi = 0; qi < KS / 4; ++qi) {
      const int q = reverse ? KS / 4 - 1 - qi : qi;
      uint32_t a[8][4];
      if (MODE == 0) {
        // replicated words, 128-byte swizzled rows of 32 words
        const uint32_t *Aw = reinterpret_cast<const uint32_t *>(As + st * A_BYTES) + ty * KS;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint4 v = *reinterpret_cast<const uint4 *>(Aw + G * r * KS + ((q ^ (ty & 7)) << 2));
          a[r][0] = v.x; a[r][1] = v.y; a[r][2] = v.z; a[r][3] = v.w;
        }
      } else {
        // int16 rows of 32 k's (64 bytes): 4 k's = one 64-bit load
        const int16_t *Ah = reinterpret_cast<const int16_t *>(As + st * A_BYTES) + ty * KS;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const uint2 v = *reinterpret_cast<const uint2 *>(Ah + G * r * KS + 4 * q);
          a[r][0] = rep_lo(v.x); a[r][1] = rep_hi(v.x); a[r][2] = rep_lo(v.y); a[r][3] = rep_hi(v.y);
        }
      }
#pragma unroll
      for (int ui = 0; ui < 4; ++ui) {
        const int u = reverse ? 3 - ui : ui;
        const uint4 bv = *reinterpret_cast<const uint4 *>(Bw + (4 * q + u) * (S / 2));
        const uint32_t bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int m = 0; m < 4; ++m) acc[r][m] = __viaddmin_s16x2(a[r][u], bb[m], acc[r][m]);
      }
    }
    // the last warp done with stage st refills it (no CTA barrier per slice)
    if (s + P::STAGES < P::NSL)
      ring_release<P::STAGES, P::TPB / 32>(ring, st, timed_out, [&] { issue(s + P::STAGES, st); });
  }
  // one barrier per tile: every slice consumed, and (deferred form) the C
  // tile arrived
  const bool c_late = DEFER_C && !timed_out && !mbar_wait_bounded(cbar, 0);
  if (__syncthreads_or(timed_out || c_late)) {
    if (tid == 0) {
      ring_drain(ring, full, err);
      if (DEFER_C) mbar_wait_bounded(cbar, 0);
    }
    return;
  }

  if (DEFER_C) {
    // fold in the C tile (rows ty + G r, int16 columns 8 tx .. 8 tx + 7)
    const int64_t vi0 = (int64_t)lds_volatile(tile_ij) * S, vj0 = (int64_t)lds_volatile(tile_ij + 1) * S;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint4 c = *reinterpret_cast<const uint4 *>(Cs + (ty + G * r) * (S * 2) + 16 * tx);
      const uint32_t cw[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (VIA && via) {  // path bookkeeping: the k-block result against the tile's value
          const int64_t gi = vi0 + ty + G * r, gj = vj0 + 8 * tx + 2 * m;
          if (gi < n && gj < n) note_via(via, via_ld, gi, gj, (int)(int16_t)(acc[r][m] & 0xffffu),
                                          (int)(int16_t)(cw[m] & 0xffffu), b);
          if (gi < n && gj + 1 < n) note_via(via, via_ld, gi, gj + 1, (int)(int16_t)(acc[r][m] >> 16),
                                              (int)(int16_t)(cw[m] >> 16), b);
        }
        acc[r][m] = __vmins2(acc[r][m], cw[m]);
      }
    }
  }

  // tile coordinates from shared memory: nothing of them stays live in
  // registers across the main loop
  It = lds_volatile(tile_ij);
  Jt = lds_volatile(tile_ij + 1);
  I0 = (int64_t)It * S;
  J0 = (int64_t)Jt * S;
  const bool full_tile_out = I0 + S <= n && J0 + S <= n;
  const bool col_panel = MODE == 1 && It != b;
  if (!DEFER_C && VIA && via) {  // path bookkeeping: compare with the values about to be replaced
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int64_t gi = I0 + ty + G * r, gj = J0 + 8 * tx + 2 * m + e;
          if (gi < n && gj < n)
            note_via(via, via_ld, gi, gj, (int)(int16_t)(e ? acc[r][m] >> 16 : acc[r][m] & 0xffffu),
                     (int)d[gi * ld + gj], b);
        }
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t gi = I0 + ty + G * r;
    const int64_t gj = J0 + 8 * tx;
    if (full_tile_out) {
      *reinterpret_cast<uint4 *>(d + gi * ld + gj) = make_uint4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
    } else {
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        if (gi < n && gj + 2 * m < n) d[gi * ld + gj + 2 * m] = (int16_t)(acc[r][m] & 0xffffu);
        if (gi < n && gj + 2 * m + 1 < n) d[gi * ld + gj + 2 * m + 1] = (int16_t)(acc[r][m] >> 16);
      }
    }
  }
  if (MODE == 1 && col_panel) {
    // replicated copy of the updated column panel tile: arep[row * S + k]
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int64_t row = I0 + ty + G * r;
      uint32_t w[8];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        w[2 * m] = rep_lo(acc[r][m]);
        w[2 * m + 1] = rep_hi(acc[r][m]);
      }
      uint4 *dst = reinterpret_cast<uint4 *>(arep + row * S + 8 * tx);
      dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
      dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    }
  }
}

}  // namespace apsp
