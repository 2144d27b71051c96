// Host loop over the stages of Fig. 2 (one stage per k-block b): phase 1,
// phase 2 and phase 3 are stream-ordered launches, as in Sec. 3.2, with an
// optional lookahead that overlaps the next stage's phases 1 and 2 with the
// bulk of phase 3.
#pragma once

#include "../../include/apsp.h"
#include "apsp_internal.h"
#include "fw_kernels.cuh"
#include "fw_s16x2.cuh"

#include <type_traits>

namespace apsp {

template <typename T> struct TmaType;
template <> struct TmaType<int32_t> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_INT32; };
template <> struct TmaType<float> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };

// Tensor maps of the packed int16x2 path: the int16 matrix for the A box
// (32 k's x S rows) and the B box (S columns x 32 k's), and the replicated
// column panel in the workspace (S words x n_p rows, 128-byte swizzle).
template <int S>
static bool make_s16_maps(int16_t *d, int64_t n, int64_t ld, uint32_t *arep, int64_t np, CUtensorMap *mA16,
                          CUtensorMap *mB16, CUtensorMap *mArep, CUtensorMap *mC16) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint32_t estr[2] = {1, 1};
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(int16_t)};
  const cuuint32_t boxA[2] = {(cuuint32_t)P3S16<S>::KS, (cuuint32_t)S};
  const cuuint32_t boxB[2] = {(cuuint32_t)S, (cuuint32_t)P3S16<S>::KS};
  if (enc(mA16, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, d, dims, strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  if (enc(mB16, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, d, dims, strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint32_t boxC[2] = {(cuuint32_t)S, (cuuint32_t)S};  // the whole C tile (deferred form)
  if (enc(mC16, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, d, dims, strides, boxC, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t rdims[2] = {(cuuint64_t)S, (cuuint64_t)np};
  const cuuint64_t rstr[1] = {(cuuint64_t)S * sizeof(uint32_t)};
  const cuuint32_t rbox[2] = {(cuuint32_t)P3S16<S>::KS, (cuuint32_t)S};
  return enc(mArep, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, arep, rdims, rstr, rbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the matrix for the two panel boxes of phase 3.
template <typename T, int S>
static bool make_panel_maps(T *d, int64_t n, int64_t ld, CUtensorMap *mA, CUtensorMap *mB) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * sizeof(T)};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t boxA[2] = {(cuuint32_t)P3Tma<S>::KS, (cuuint32_t)S};  // 32 k's x S rows
  const cuuint32_t boxB[2] = {(cuuint32_t)S, (cuuint32_t)P3Tma<S>::KS};  // S cols x 32 k's
  if (enc(mA, TmaType<T>::v, 2, d, dims, strides, boxA, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  if (enc(mB, TmaType<T>::v, 2, d, dims, strides, boxB, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  return true;
}

// Tensor map of the k-pair interleaved row panel (S/2 rows x 2 n_p floats).
template <int S>
static bool make_interleaved_map(float *bp, int64_t np, CUtensorMap *m) {
  EncodeTiledFn enc = encode_tiled_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)(2 * np), (cuuint64_t)(S / 2)};
  const cuuint64_t strides[1] = {(cuuint64_t)(2 * np) * sizeof(float)};
  const cuuint32_t estr[2] = {1, 1};
  const cuuint32_t box[2] = {(cuuint32_t)(2 * S), (cuuint32_t)(P3Tma<S>::KS / 2)};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bp, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename T, int S>
struct Kernels {
  static constexpr int NT1 = (S / 4) * (S / 4);
  static constexpr int NT1_SIDE = (S / 8) * (S / 4);  // phase 1 beside phase 3
  static constexpr int NT2 = S == 64 ? 256 : 1024;
  using C = typename Arith<T>::C;
  static constexpr size_t SM2 = 2 * (size_t)S * S * sizeof(C);
  static constexpr size_t SM3G = ((size_t)S * (S + 1) + (size_t)S * S) * sizeof(C);

  // Raises the dynamic shared-memory limit of each kernel once per process
  // and device (the attribute is per device).
  static cudaError_t setup() {
    cudaError_t e;
    e = cudaFuncSetAttribute(fw_phase2<T, S, NT2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM2);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fw_phase3_generic<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM3G);
    return e;
  }
};

// Launches `k` on `st` as a programmatic dependent launch (see
// wait_prior_grid); prio != 0 sets the launch's scheduling priority (both
// are recorded in the node when the stream is being captured).
template <typename... KP, typename... Args>
static cudaError_t launch(void (*k)(KP...), dim3 grid, int threads, size_t smem, cudaStream_t st, int prio,
                          Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  unsigned na = 0;
#if APSP_PDL
  // every kernel launched here starts with wait_prior_grid()
  at[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[na].val.programmaticStreamSerializationAllowed = 1;
  ++na;
#endif
  if (prio != 0) {
    at[na].id = cudaLaunchAttributePriority;
    at[na].val.priority = prio;
    ++na;
  }
  cfg.attrs = na ? at : nullptr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

// The stages of Fig. 2 for one matrix.
//
// Plain schedule, per stage b on the caller's stream: phase 1, phase 2,
// phase 3 (all doubly dependent tiles).
//
// Lookahead schedule (R >= kLookaheadMinRounds, TMA kernels, a side stream):
// phase 3 of stage b is split into cross(b) -- row and column b+1, the tiles
// that phases 1 and 2 of stage b+1 read -- and rest(b), every other tile.
//   side stream:    cross(b), phase 1 (b+1), phase 2 (b+1)
//   caller's stream: rest(b)
// both starting once phase 2 (b) and rest(b-1) are done, and joined before
// stage b+1 continues.  rest(b) reads panel b and writes no tile of row or
// column b+1, which phase 2 (b+1) updates beside it; the panel copies that
// phase 2 writes for phase 3 (interleaved fp32 row panel, replicated int16
// column panel) alternate between two workspace buffers.  The side stream's
// launches run at a higher priority, so their CTAs take SM slots as rest(b)
// CTAs retire: the mostly serial phase 1 and the one-wave phase 2 no longer
// leave the GPU idle between the phase-3 launches.  Every tile still sees
// every stage in order, so results equal the plain schedule's bit for bit.
//
// Small matrices (uses_strips: s = 64, few stages): phase 2 and cross(b) have
// fewer tiles than SMs and sit on the stage's critical path, so they run as
// fw_strip launches, four CTAs per tile; the values are those of the TMA
// kernels.
template <typename T, int S, bool HAS_TMA, bool VIA>
static int run_rounds(const RunArgs &a) {
  using K = Kernels<T, S>;
  static thread_local uint64_t setup_done_mask = 0;  // bit per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return APSP_ECUDA;
  if (!(setup_done_mask & (1ull << dev))) {
    if (K::setup() != cudaSuccess) return APSP_ECUDA;
    if constexpr (HAS_TMA) {
      if (cudaFuncSetAttribute(fw_tile_tma<T, S, 0, VIA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P3Tma<S>::SMEM) != cudaSuccess ||
          cudaFuncSetAttribute(fw_tile_tma<T, S, 1, VIA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P3Tma<S>::SMEM) != cudaSuccess)
        return APSP_ECUDA;
      if constexpr (std::is_same<T, float>::value) {
        const int sm = P3Tma<S>::SMEM;
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(fw_phase3_f32x2<S, false, true, VIA>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, true, true, VIA>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, false, false, VIA>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, true, false, VIA>, attr, sm) != cudaSuccess)
          return APSP_ECUDA;
      }
    }
    if constexpr (std::is_same<T, int16_t>::value) {
      const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
      if (cudaFuncSetAttribute(fw_tile_s16x2<S, 0, VIA>, attr, P3S16<S>::SMEM_P3) != cudaSuccess ||
          cudaFuncSetAttribute(fw_tile_s16x2<S, 1, VIA>, attr, P3S16<S>::SMEM) != cudaSuccess)
        return APSP_ECUDA;
    }
    setup_done_mask |= 1ull << dev;
  }

  T *d = static_cast<T *>(a.d);
  const int64_t n = a.n, ld = a.ld;
  const int R = (int)((n + S - 1) / S);
  const bool ragged = (n % S) != 0;
  const int reverse = (a.flags & APSP_FLAG_REVERSE_K) ? 1 : 0;
  const bool generic_only = (a.flags & APSP_FLAG_GENERIC) != 0;

  // Small matrices, on request: all stages in one launch (same values as below).
  if constexpr (S == 64) {
    constexpr int kFlagsOff = APSP_FLAG_GENERIC | APSP_FLAG_REVERSE_K | APSP_FLAG_NO_LOOKAHEAD;
    if ((a.flags & APSP_FLAG_ONE_LAUNCH) && R >= kDataflowMinRounds && R <= kDataflowMaxRounds &&
        !(a.flags & kFlagsOff) && !a.via && !a.events && !a.first_src && !a.last_dst && a.ws &&
        a.ws_bytes >= dataflow_flag_bytes(R) && reinterpret_cast<uintptr_t>(a.ws) % 16 == 0) {
      const int dt = std::is_same<T, float>::value ? APSP_F32 : std::is_same<T, int16_t>::value ? APSP_I16 : APSP_I32;
      return run_dataflow(a, dt, static_cast<int *>(a.ws));
    }
  }
  const cudaStream_t st = a.stream;
  const int64_t np = (int64_t)R * S;

  // Tensor maps; the panel copies of phase 2 (one buffer, or two for the
  // lookahead schedule).
  CUtensorMap mA, mB, mBp[2];
  bool use_tma = false, use_packed = false;
  T *bp[2] = {nullptr, nullptr};
  int nbuf = 0;
  if constexpr (HAS_TMA) {
    use_tma = a.tma_ok && !generic_only && R > 1 && make_panel_maps<T, S>(d, n, ld, &mA, &mB);
    if constexpr (std::is_same<T, float>::value) {
      const size_t pb = interleaved_panel_bytes(n, S);
      if (use_tma && a.ws && a.ws_bytes >= pb && reinterpret_cast<uintptr_t>(a.ws) % 256 == 0) {
        nbuf = a.ws_bytes >= 2 * pb ? 2 : 1;
        use_packed = true;
        for (int i = 0; i < nbuf; ++i) {
          bp[i] = reinterpret_cast<T *>(static_cast<char *>(a.ws) + i * pb);
          use_packed = use_packed && make_interleaved_map<S>(reinterpret_cast<float *>(bp[i]), np, &mBp[i]);
        }
        if (!use_packed) nbuf = 0;
      }
    }
  }

  CUtensorMap mA16, mB16, mC16, mArep[2];
  bool use_s16 = false;
  uint32_t *arep[2] = {nullptr, nullptr};
  if constexpr (std::is_same<T, int16_t>::value) {
    const size_t pb = replicated_panel_bytes(n, S);
    if (a.tma_ok && !generic_only && R > 1 && a.ws && a.ws_bytes >= pb &&
        reinterpret_cast<uintptr_t>(a.ws) % 256 == 0) {
      nbuf = a.ws_bytes >= 2 * pb ? 2 : 1;
      use_s16 = true;
      for (int i = 0; i < nbuf; ++i) {
        arep[i] = reinterpret_cast<uint32_t *>(static_cast<char *>(a.ws) + i * pb);
        use_s16 = use_s16 && make_s16_maps<S>(reinterpret_cast<int16_t *>(d), n, ld, arep[i], np, &mA16, &mB16,
                                              &mArep[i], &mC16);
      }
      if (!use_s16) nbuf = 0;
    }
  }

  // Is phase 3 of a full stage done by a TMA kernel (tile sets supported)?
  bool p3_tma = false;
  if constexpr (std::is_same<T, int16_t>::value) p3_tma = use_s16;
  else p3_tma = use_tma;
  const bool needs_panel = use_packed || use_s16;
  // A caller that supplies its workspace for the packed fp32 kernels (the
  // allocation-free entry point) is told when they cannot run on it, before
  // any work is enqueued, instead of getting the unpacked kernels silently.
  if constexpr (std::is_same<T, float>::value) {
    if (a.require_ws && a.tma_ok && !generic_only && R > 1 && !use_packed) return APSP_EUNSUPPORTED;
  }
  const bool routed = a.first_src || a.last_dst;
  const auto aligned16 = [](const void *p, int64_t ld_) {
    return reinterpret_cast<uintptr_t>(p) % 16 == 0 && ((size_t)ld_ * sizeof(T)) % 16 == 0;
  };
  if (routed && (ragged || R < 2 || !p3_tma || std::is_same<T, int16_t>::value ||
                 (a.first_src && !aligned16(a.first_src, a.first_src_ld)) ||
                 (a.last_dst && !aligned16(a.last_dst, a.last_dst_ld))))
    return APSP_EUNSUPPORTED;
  const bool lookahead = p3_tma && a.side && !(a.flags & APSP_FLAG_NO_LOOKAHEAD) && R >= kLookaheadMinRounds &&
                         (!needs_panel || nbuf == 2);
  auto buf_of = [&](int b) { return lookahead ? (b & 1) : 0; };
  const bool strips = uses_strips(S, R, std::is_same<T, float>::value, std::is_same<T, int16_t>::value);

  auto ev = [&](int64_t idx, cudaStream_t s) -> bool {
    if (!a.events || idx >= a.n_events) return true;
    return cudaEventRecord(static_cast<cudaEvent_t>(a.events[idx]), s) == cudaSuccess;
  };
  auto full_k = [&](int b) { return (int64_t)(b + 1) * S <= n; };

  // ---- the three phases of one stage, on stream s with priority prio
  auto phase1 = [&](int b, cudaStream_t s, int prio) -> cudaError_t {
    const int last = b == R - 1 ? 1 : 0;
    if (prio != 0)
      return launch(fw_phase1_side<T, S>, dim3(1), K::NT1_SIDE, 0, s, prio, d, n, ld, b, last, a.via, a.via_ld);
    return launch(fw_phase1<T, S>, dim3(1), K::NT1, 0, s, 0, d, n, ld, b, last, a.via, a.via_ld);
  };
  auto phase2 = [&](int b, cudaStream_t s, int prio) -> cudaError_t {
    if (R == 1) return cudaSuccess;
    const int last = b == R - 1 ? 1 : 0;
    const dim3 g(2 * (R - 1));
    if constexpr (std::is_same<T, int16_t>::value) {
      if (use_s16 && full_k(b))
        return launch(fw_tile_s16x2<S, 1, VIA>, g, P3S16<S>::TPB, P3S16<S>::SMEM, s, prio, mA16, mB16, mC16,
                      reinterpret_cast<int16_t *>(d), n, ld, b, R, TileSet{}, reverse, arep[buf_of(b)], a.via,
                      a.via_ld, a.err);
    }
    T *bpb = (use_packed && full_k(b)) ? bp[buf_of(b)] : nullptr;
    if constexpr (HAS_TMA && S == 64 && !std::is_same<T, int16_t>::value) {
      // four strips per panel tile while the stage is latency bound
      if (use_tma && full_k(b) && strips)
        return launch(fw_strip<T, S, 1, VIA>, dim3(8 * (R - 1)), 64, 0, s, prio, CRoute<T>{d, ld, d, ld},
                      (const T *)d, n, ld, b, R, TileSet{}, last, reverse, bpb, 2 * np, a.via, a.via_ld);
    }
    if constexpr (HAS_TMA) {
      if (use_tma && full_k(b))
        return launch(fw_tile_tma<T, S, 1, VIA>, g, P3Tma<S>::TPB, P3Tma<S>::SMEM, s, prio, mA, mB,
                      CRoute<T>{d, ld, d, ld}, n, b, R, TileSet{}, last, reverse, bpb, 2 * np, a.via, a.via_ld,
                      a.err);
    }
    return launch(fw_phase2<T, S, K::NT2>, g, K::NT2, K::SM2, s, prio, d, n, ld, b, R, last, bpb, 2 * np, a.via,
                  a.via_ld);
  };
  // phase 3 of stage b over the tiles of `kind`
  auto phase3 = [&](int b, int kind, cudaStream_t s, int prio) -> cudaError_t {
    if (R == 1) return cudaSuccess;
    const int last = b == R - 1 ? 1 : 0;
    CRoute<T> cr{d, ld, d, ld};
    if (b == 0 && a.first_src) {
      cr.src = static_cast<const T *>(a.first_src);
      cr.src_ld = a.first_src_ld;
    }
    if (last && a.last_dst) {
      cr.dst = static_cast<T *>(a.last_dst);
      cr.dst_ld = a.last_dst_ld;
    }
    if (full_k(b)) {
      if constexpr (HAS_TMA && S == 64 && !std::is_same<T, int16_t>::value) {
        // the cross tiles of the lookahead schedule: as few as the panel
        // tiles and on the critical path, so cut into strips as well
        if (kind == kTilesCross && use_tma && strips) {
          const TileSet ts = make_tileset(kind, kPartAny, b, R, ragged);
          if (ts.total() == 0) return cudaSuccess;
          return launch(fw_strip<T, S, 0, VIA>, dim3(4 * ts.total()), 64, 0, s, prio, cr, (const T *)d, n, ld, b,
                        R, ts, last, reverse, (T *)nullptr, (int64_t)0, a.via, a.via_ld);
        }
      }
      if constexpr (std::is_same<T, int16_t>::value) {
        if (use_s16) {
          const TileSet ts = make_tileset(kind, kPartAny, b, R, ragged);
          if (ts.total() == 0) return cudaSuccess;
          return launch(fw_tile_s16x2<S, 0, VIA>, dim3(ts.total()), P3S16<S>::TPB, P3S16<S>::SMEM_P3, s, prio,
                        mArep[buf_of(b)], mB16, mC16, reinterpret_cast<int16_t *>(d), n, ld, b, R, ts, reverse,
                        arep[buf_of(b)], a.via, a.via_ld, a.err);
        }
      }
      if constexpr (std::is_same<T, float>::value) {
        if (use_packed) {
          const int tpb = P3Tma<S>::TPB, sm = P3Tma<S>::SMEM;
          const CUtensorMap &mb = mBp[buf_of(b)];
          const TileSet ti = make_tileset(kind, kPartInterior, b, R, ragged);
          const TileSet te = make_tileset(kind, kPartEdge, b, R, ragged);
          cudaError_t e = cudaSuccess;
          if (ti.total() > 0)
            e = reverse ? launch(fw_phase3_f32x2<S, true, true, VIA>, dim3(ti.total()), tpb, sm, s, prio, mA, mb,
                                 cr, n, b, ti, a.via, a.via_ld, a.err)
                        : launch(fw_phase3_f32x2<S, false, true, VIA>, dim3(ti.total()), tpb, sm, s, prio, mA, mb,
                                 cr, n, b, ti, a.via, a.via_ld, a.err);
          if (e == cudaSuccess && te.total() > 0)
            e = reverse ? launch(fw_phase3_f32x2<S, true, false, VIA>, dim3(te.total()), tpb, sm, s, prio, mA, mb,
                                 cr, n, b, te, a.via, a.via_ld, a.err)
                        : launch(fw_phase3_f32x2<S, false, false, VIA>, dim3(te.total()), tpb, sm, s, prio, mA, mb,
                                 cr, n, b, te, a.via, a.via_ld, a.err);
          return e;
        }
      }
      if constexpr (HAS_TMA) {
        if (use_tma) {
          const TileSet ts = make_tileset(kind, kPartAny, b, R, ragged);
          if (ts.total() == 0) return cudaSuccess;
          return launch(fw_tile_tma<T, S, 0, VIA>, dim3(ts.total()), P3Tma<S>::TPB, P3Tma<S>::SMEM, s, prio, mA, mB, cr,
                        n, b, R, ts, last, reverse, (T *)nullptr, (int64_t)0, a.via, a.via_ld, a.err);
        }
      }
    }
    // generic kernel: all tiles of the stage (plain schedule only)
    return launch(fw_phase3_generic<T, S>, dim3(R - 1, R - 1), 256, K::SM3G, s, prio, d, n, ld, b, last,
                  reverse, a.via, a.via_ld);
  };

  const int E = kEventsPerStage;
  auto stage_12 = [&](int b, cudaStream_t s, int prio) -> bool {
    return ev((int64_t)E * b, s) && phase1(b, s, prio) == cudaSuccess && ev((int64_t)E * b + 1, s) &&
           phase2(b, s, prio) == cudaSuccess && ev((int64_t)E * b + 2, s);
  };

  if (!stage_12(0, st, 0)) return APSP_ECUDA;
  for (int b = 0; b < R; ++b) {
    if (lookahead && b + 1 < R) {
      // b + 1 < R implies a full k-block for stage b
      if (cudaEventRecord(a.fork, st) != cudaSuccess || cudaStreamWaitEvent(a.side, a.fork, 0) != cudaSuccess)
        return APSP_ECUDA;
      if (phase3(b, kTilesCross, a.side, a.side_prio) != cudaSuccess) return APSP_ECUDA;
      if (!stage_12(b + 1, a.side, a.side_prio)) return APSP_ECUDA;
      if (cudaEventRecord(a.join, a.side) != cudaSuccess) return APSP_ECUDA;
      if (!ev((int64_t)E * b + 3, st) || phase3(b, kTilesRest, st, 0) != cudaSuccess ||
          !ev((int64_t)E * b + 4, st))
        return APSP_ECUDA;
      if (cudaStreamWaitEvent(st, a.join, 0) != cudaSuccess) return APSP_ECUDA;
    } else {
      if (!ev((int64_t)E * b + 3, st) || phase3(b, kTilesAll, st, 0) != cudaSuccess || !ev((int64_t)E * b + 4, st))
        return APSP_ECUDA;
      if (b + 1 < R && !stage_12(b + 1, st, 0)) return APSP_ECUDA;
    }
    if (cudaPeekAtLastError() != cudaSuccess) return APSP_ECUDA;
  }
  return APSP_OK;
}

template <typename T, bool HAS_TMA>
static int run_any(const RunArgs &a) {
  if (a.n == 0) return APSP_OK;
  switch (a.S) {
    case 64: return a.via ? run_rounds<T, 64, HAS_TMA, true>(a) : run_rounds<T, 64, HAS_TMA, false>(a);
    case 128: return a.via ? run_rounds<T, 128, HAS_TMA, true>(a) : run_rounds<T, 128, HAS_TMA, false>(a);
    default: return APSP_EINVAL;
  }
}

}  // namespace apsp
