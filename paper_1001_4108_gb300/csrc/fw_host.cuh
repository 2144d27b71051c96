// Host loop over the stages of Fig. 2 (one stage per k-block b): phase 1,
// phase 2 and phase 3 are three stream-ordered launches, as in Sec. 3.2.
#pragma once

#include "../../include/apsp.h"
#include "apsp_internal.h"
#include "fw_kernels.cuh"

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
                          CUtensorMap *mB16, CUtensorMap *mArep) {
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

template <typename T, int S, bool HAS_TMA>
static int run_rounds(const RunArgs &a) {
  using K = Kernels<T, S>;
  static thread_local int setup_done_mask = 0;  // bit per device
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
  if (!(setup_done_mask & (1 << (dev & 31)))) {
    if (K::setup() != cudaSuccess) return APSP_ECUDA;
    if constexpr (HAS_TMA) {
      if (cudaFuncSetAttribute(fw_tile_tma<T, S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P3Tma<S>::SMEM) != cudaSuccess ||
          cudaFuncSetAttribute(fw_tile_tma<T, S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P3Tma<S>::SMEM) != cudaSuccess)
        return APSP_ECUDA;
      if constexpr (std::is_same<T, float>::value) {
        const int sm = P3Tma<S>::SMEM;
        const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (cudaFuncSetAttribute(fw_phase3_f32x2<S, false, true>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, true, true>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, false, false>, attr, sm) != cudaSuccess ||
            cudaFuncSetAttribute(fw_phase3_f32x2<S, true, false>, attr, sm) != cudaSuccess)
          return APSP_ECUDA;
      }
    }
    if constexpr (std::is_same<T, int16_t>::value) {
      const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
      if (cudaFuncSetAttribute(fw_tile_s16x2<S, 0>, attr, P3S16<S>::SMEM) != cudaSuccess ||
          cudaFuncSetAttribute(fw_tile_s16x2<S, 1>, attr, P3S16<S>::SMEM) != cudaSuccess)
        return APSP_ECUDA;
    }
    setup_done_mask |= 1 << (dev & 31);
  }

  T *d = static_cast<T *>(a.d);
  const int64_t n = a.n, ld = a.ld;
  const int R = (int)((n + S - 1) / S);
  const int reverse = (a.flags & APSP_FLAG_REVERSE_K) ? 1 : 0;
  const bool generic_only = (a.flags & APSP_FLAG_GENERIC) != 0;
  cudaStream_t st = a.stream;

  CUtensorMap mA, mB, mBp;
  bool use_tma = false, use_packed = false;
  T *bp = nullptr;
  const int64_t np = (int64_t)R * S;
  if constexpr (HAS_TMA) {
    use_tma = a.tma_ok && !generic_only && R > 1 && make_panel_maps<T, S>(d, n, ld, &mA, &mB);
    if constexpr (std::is_same<T, float>::value) {
      use_packed = use_tma && a.ws && a.ws_bytes >= interleaved_panel_bytes(n, S) &&
                   reinterpret_cast<uintptr_t>(a.ws) % 256 == 0 &&
                   make_interleaved_map<S>(static_cast<float *>(a.ws), np, &mBp);
      if (use_packed) bp = static_cast<T *>(a.ws);
    }
  }

  CUtensorMap mA16, mB16, mArep;
  bool use_s16 = false;
  uint32_t *arep = nullptr;
  if constexpr (std::is_same<T, int16_t>::value) {
    arep = static_cast<uint32_t *>(a.ws);
    use_s16 = a.tma_ok && !generic_only && R > 1 && a.ws && a.ws_bytes >= replicated_panel_bytes(n, S) &&
              reinterpret_cast<uintptr_t>(a.ws) % 256 == 0 &&
              make_s16_maps<S>(reinterpret_cast<int16_t *>(d), n, ld, arep, np, &mA16, &mB16, &mArep);
  }

  auto ev = [&](int64_t idx) -> bool {
    if (!a.events || idx >= a.n_events) return true;
    return cudaEventRecord(static_cast<cudaEvent_t>(a.events[idx]), st) == cudaSuccess;
  };

  for (int b = 0; b < R; ++b) {
    const int last = (b == R - 1) ? 1 : 0;
    if (!ev(4ll * b)) return APSP_ECUDA;
    fw_phase1<T, S><<<1, K::NT1, 0, st>>>(d, n, ld, b, last);
    if (!ev(4ll * b + 1)) return APSP_ECUDA;
    const bool full_k = (int64_t)(b + 1) * S <= n;
    T *bp_round = (use_packed && full_k) ? bp : nullptr;
    if (R > 1) {
      bool launched2 = false;
      if constexpr (std::is_same<T, int16_t>::value) {
        if (use_s16 && full_k) {
          fw_tile_s16x2<S, 1><<<2 * (R - 1), P3S16<S>::TPB, P3S16<S>::SMEM, st>>>(
              mA16, mB16, reinterpret_cast<int16_t *>(d), n, ld, b, R, reverse, arep, a.err);
          launched2 = true;
        }
      }
      if constexpr (HAS_TMA) {
        if (use_tma && full_k) {
          fw_tile_tma<T, S, 1><<<2 * (R - 1), P3Tma<S>::TPB, P3Tma<S>::SMEM, st>>>(
              mA, mB, d, n, ld, b, R, last, reverse, bp_round, 2 * np, a.err);
          launched2 = true;
        }
      }
      if (!launched2)
        fw_phase2<T, S, K::NT2><<<2 * (R - 1), K::NT2, K::SM2, st>>>(d, n, ld, b, R, last, bp_round, 2 * np);
    }
    if (!ev(4ll * b + 2)) return APSP_ECUDA;
    if (R > 1) {
      const dim3 grid(R - 1, R - 1);
      bool launched = false;
      if constexpr (std::is_same<T, int16_t>::value) {
        if (use_s16 && full_k) {
          fw_tile_s16x2<S, 0><<<grid, P3S16<S>::TPB, P3S16<S>::SMEM, st>>>(
              mArep, mB16, reinterpret_cast<int16_t *>(d), n, ld, b, R, reverse, arep, a.err);
          launched = true;
        }
      }
      if constexpr (std::is_same<T, float>::value) {
        if (bp_round) {
          // interior tiles (all rows/columns inside the matrix), then the
          // edge tiles of a ragged matrix
          const int ragged = (n % S) != 0 ? 1 : 0;
          const dim3 gi(R - 1 - ragged, R - 1 - ragged);
          const int ne = ragged ? 2 * R - 3 : 0;
          const int tpb = P3Tma<S>::TPB, sm = P3Tma<S>::SMEM;
          if (gi.x > 0) {
            if (reverse)
              fw_phase3_f32x2<S, true, true><<<gi, tpb, sm, st>>>(mA, mBp, d, n, ld, b, R, a.err);
            else
              fw_phase3_f32x2<S, false, true><<<gi, tpb, sm, st>>>(mA, mBp, d, n, ld, b, R, a.err);
          }
          if (ne > 0) {
            if (reverse)
              fw_phase3_f32x2<S, true, false><<<ne, tpb, sm, st>>>(mA, mBp, d, n, ld, b, R, a.err);
            else
              fw_phase3_f32x2<S, false, false><<<ne, tpb, sm, st>>>(mA, mBp, d, n, ld, b, R, a.err);
          }
          launched = true;
        }
      }
      if constexpr (HAS_TMA) {
        if (!launched && use_tma && full_k) {
          fw_tile_tma<T, S, 0><<<grid, P3Tma<S>::TPB, P3Tma<S>::SMEM, st>>>(mA, mB, d, n, ld, b, R, last, reverse,
                                                                            (T *)nullptr, 0, a.err);
          launched = true;
        }
      }
      if (!launched) fw_phase3_generic<T, S><<<grid, 256, K::SM3G, st>>>(d, n, ld, b, last, reverse);
    }
    if (!ev(4ll * b + 3)) return APSP_ECUDA;
    if (cudaPeekAtLastError() != cudaSuccess) return APSP_ECUDA;
  }
  return APSP_OK;
}

template <typename T, bool HAS_TMA>
static int run_any(const RunArgs &a) {
  if (a.n == 0) return APSP_OK;
  switch (a.S) {
    case 64: return run_rounds<T, 64, HAS_TMA>(a);
    case 128: return run_rounds<T, 128, HAS_TMA>(a);
    default: return APSP_EINVAL;
  }
}

}  // namespace apsp
