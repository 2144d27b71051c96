// Host loop over the stages of Fig. 2 (one stage per k-block b): phase 1,
// phase 2 and phase 3 are three stream-ordered launches, as in Sec. 3.2.
#pragma once

#include "../../include/apsp.h"
#include "apsp_internal.h"
#include "fw_kernels.cuh"

namespace apsp {

template <typename T> struct TmaType;
template <> struct TmaType<int32_t> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_INT32; };
template <> struct TmaType<float> { static constexpr CUtensorMapDataType v = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; };

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

template <typename T, int S>
struct Kernels {
  static constexpr int NT12 = S == 64 ? 256 : 1024;
  using C = typename Arith<T>::C;
  static constexpr size_t SM1 = (size_t)S * S * sizeof(C);
  static constexpr size_t SM2 = 2 * SM1;
  static constexpr size_t SM3G = ((size_t)S * (S + 1) + (size_t)S * S) * sizeof(C);

  // Raises the dynamic shared-memory limit of each kernel once per process
  // and device (the attribute is per device).
  static cudaError_t setup() {
    cudaError_t e;
    e = cudaFuncSetAttribute(fw_phase1<T, S, NT12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM1);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(fw_phase2<T, S, NT12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SM2);
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
      if (cudaFuncSetAttribute(fw_phase3_tma<T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               P3Tma<S>::SMEM) != cudaSuccess)
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

  CUtensorMap mA, mB;
  bool use_tma = false;
  if constexpr (HAS_TMA) {
    use_tma = a.tma_ok && !generic_only && R > 1 && make_panel_maps<T, S>(d, n, ld, &mA, &mB);
  }

  auto ev = [&](int64_t idx) -> bool {
    if (!a.events || idx >= a.n_events) return true;
    return cudaEventRecord(static_cast<cudaEvent_t>(a.events[idx]), st) == cudaSuccess;
  };

  for (int b = 0; b < R; ++b) {
    const int last = (b == R - 1) ? 1 : 0;
    if (!ev(4ll * b)) return APSP_ECUDA;
    fw_phase1<T, S, K::NT12><<<1, K::NT12, K::SM1, st>>>(d, n, ld, b, last);
    if (!ev(4ll * b + 1)) return APSP_ECUDA;
    if (R > 1) fw_phase2<T, S, K::NT12><<<2 * (R - 1), K::NT12, K::SM2, st>>>(d, n, ld, b, R, last);
    if (!ev(4ll * b + 2)) return APSP_ECUDA;
    if (R > 1) {
      const dim3 grid(R - 1, R - 1);
      const bool full_k = (int64_t)(b + 1) * S <= n;
      bool launched = false;
      if constexpr (HAS_TMA) {
        if (use_tma && full_k) {
          fw_phase3_tma<T, S><<<grid, P3Tma<S>::TPB, P3Tma<S>::SMEM, st>>>(mA, mB, d, n, ld, b, last, reverse,
                                                                           a.err);
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
