// Roofline calibration for the min-plus relaxation (apsp_ubench_minplus).
//
// Each form runs the phase-3 inner loop of one element type on operands that
// come from shared memory every k step, exactly as in the kernels: 256
// threads, an 8 x 8 register micro-tile per thread, a 32-k slice of the two
// panels (A: 128 rows x 32 k's with 128-byte swizzled rows, B: 32 k's x 128
// columns, or 16 k-pairs x 256 interleaved floats for the packed fp32 form),
// swept `iters` times.  Real loads matter: register-only loops let the
// compiler hoist the additions out of the loop and measure the minimum alone.
// Relaxations per second divided by SMs x clock give relaxations per clock
// per SM for each instruction form.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apsp.h"

namespace {

constexpr int kRows = 128, kKs = 32, kCols = 128;

__device__ __forceinline__ int32_t relax_dpx(int32_t acc, int32_t a, int32_t b) { return __viaddmin_s32(a, b, acc); }
__device__ __forceinline__ int32_t relax_addmin(int32_t acc, int32_t a, int32_t b) {
  int32_t s, r;
  asm volatile("add.s32 %0, %1, %2;" : "=r"(s) : "r"(a), "r"(b));
  asm volatile("min.s32 %0, %1, %2;" : "=r"(r) : "r"(acc), "r"(s));
  return r;
}
__device__ __forceinline__ float relax_f32(float acc, float a, float b) { return fminf(acc, __fadd_rn(a, b)); }
__device__ __forceinline__ uint32_t relax_s16x2(uint32_t acc, uint32_t a, uint32_t b) {
  return __viaddmin_s16x2(a, b, acc);
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

template <typename T> __device__ __forceinline__ T fill(int i);
template <> __device__ __forceinline__ int32_t fill<int32_t>(int i) { return i % 997; }
template <> __device__ __forceinline__ uint32_t fill<uint32_t>(int i) { return (uint32_t)(i % 991) * 0x10001u; }
template <> __device__ __forceinline__ float fill<float>(int i) { return (float)(i % 997) * 0.001f; }

// forms 0, 1, 2, 3: one k per step (the integer / unpacked kernels' loop:
// k-quads of A by 128-bit loads, two 128-bit loads of B per k).
template <typename T, int FORM>
__global__ void __launch_bounds__(256, 2) ubench_kstep(int64_t iters, T *sink) {
  __shared__ __align__(16) T As[kRows * kKs];
  __shared__ __align__(16) T Bs[kKs * kCols];
  for (int i = threadIdx.x; i < kRows * kKs; i += blockDim.x) As[i] = fill<T>(i);
  for (int i = threadIdx.x; i < kKs * kCols; i += blockDim.x) Bs[i] = fill<T>(i + 7);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16, sw = ty & 7;
  const T *A = As + ty * kKs;
  const T *B = Bs + 4 * tx;
  T acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = fill<T>(1000 + r + c);
#pragma unroll 1
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 2
    for (int q = 0; q < kKs / 4; ++q) {
      T a[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const uint4 v = *reinterpret_cast<const uint4 *>(A + 16 * r * kKs + ((q ^ sw) << 2));
        a[r][0] = __builtin_bit_cast(T, v.x);
        a[r][1] = __builtin_bit_cast(T, v.y);
        a[r][2] = __builtin_bit_cast(T, v.z);
        a[r][3] = __builtin_bit_cast(T, v.w);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint4 b0 = *reinterpret_cast<const uint4 *>(B + (4 * q + u) * kCols);
        const uint4 b1 = *reinterpret_cast<const uint4 *>(B + (4 * q + u) * kCols + kCols / 2);
        const T bv[8] = {__builtin_bit_cast(T, b0.x), __builtin_bit_cast(T, b0.y), __builtin_bit_cast(T, b0.z),
                         __builtin_bit_cast(T, b0.w), __builtin_bit_cast(T, b1.x), __builtin_bit_cast(T, b1.y),
                         __builtin_bit_cast(T, b1.z), __builtin_bit_cast(T, b1.w)};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            if constexpr (FORM == 0) acc[r][c] = relax_dpx(acc[r][c], a[r][u], bv[c]);
            if constexpr (FORM == 1) acc[r][c] = relax_f32(acc[r][c], a[r][u], bv[c]);
            if constexpr (FORM == 2) acc[r][c] = relax_s16x2(acc[r][c], a[r][u], bv[c]);
            if constexpr (FORM == 3) acc[r][c] = relax_addmin(acc[r][c], a[r][u], bv[c]);
          }
      }
    }
  }
  T s = acc[0][0];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s = acc[r][c] < s ? acc[r][c] : s;
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// form 9: the int16x2 phase-3 loop as the kernel runs it: an 8 x 4 word
// micro-tile (8 rows x 8 int16 columns), A k-quads of replicated words by
// 128-bit loads, one 128-bit load of B (rows of 64 words) per k.
__global__ void __launch_bounds__(256, 2) ubench_s16x2_narrow(int64_t iters, uint32_t *sink) {
  constexpr int kWords = kCols / 2;  // a B row: 128 int16 columns
  __shared__ __align__(16) uint32_t As[kRows * kKs];
  __shared__ __align__(16) uint32_t Bs[kKs * kWords];
  for (int i = threadIdx.x; i < kRows * kKs; i += blockDim.x) As[i] = fill<uint32_t>(i);
  for (int i = threadIdx.x; i < kKs * kWords; i += blockDim.x) Bs[i] = fill<uint32_t>(i + 7);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16, sw = ty & 7;
  const uint32_t *A = As + ty * kKs;
  const uint32_t *B = Bs + 4 * tx;
  uint32_t acc[8][4];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = fill<uint32_t>(1000 + r + c);
#pragma unroll 1
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 2
    for (int q = 0; q < kKs / 4; ++q) {
      uint32_t a[8][4];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const uint4 v = *reinterpret_cast<const uint4 *>(A + 16 * r * kKs + ((q ^ sw) << 2));
        a[r][0] = v.x; a[r][1] = v.y; a[r][2] = v.z; a[r][3] = v.w;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint4 bv = *reinterpret_cast<const uint4 *>(B + (4 * q + u) * kWords);
        const uint32_t bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[r][c] = relax_s16x2(acc[r][c], a[r][u], bb[c]);
      }
    }
  }
  uint32_t s = acc[0][0];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) s = acc[r][c] < s ? acc[r][c] : s;
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// form 4: the packed fp32 loop: per k-pair, 8 (k, k+1) pairs of A (64-bit
// loads) and 4 column-pair quads of the k-pair interleaved B (128-bit loads),
// then acc <- min(acc, a_k + b_k, a_k' + b_k') with one add.f32x2 and one
// three-input min per (row, column).
// form 5: int32, two adds + one three-input minimum per (row, column, k-pair).
// form 6: fp32, two scalar adds + one three-input minimum per (row, column,
// k-pair) (the adds may issue on either FMA sub-pipe).
// form 8: int32, additions split between the pipes -- three of every four as
// a multiply-add by a runtime 1 (FMA pipe), one as an add (ALU) -- and one
// three-input DPX minimum per (row, column, k-pair).
// form 7: fp32, the two forms alternating by column: one packed add for
// column 2m, two scalar adds for column 2m + 1.
template <int FORM>
__global__ void __launch_bounds__(256, 2) ubench_kpair(int64_t iters, void *sinkv) {
  __shared__ __align__(16) float As[kRows * kKs];
  __shared__ __align__(16) float Bs[(kKs / 2) * 2 * kCols];
  for (int i = threadIdx.x; i < kRows * kKs; i += blockDim.x) As[i] = fill<float>(i);
  for (int i = threadIdx.x; i < kKs * kCols; i += blockDim.x) Bs[i] = fill<float>(i + 7);
  __syncthreads();
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16, sw = ty & 7;
  const float *A = As + ty * kKs;
  const float *B = Bs + 4 * tx;
  float acc[8][8];
  int32_t iacc[8][8];
  const int32_t one = iters > 0 ? 1 : 0;  // a 1 the compiler cannot fold away
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      acc[r][c] = 1e20f;
      iacc[r][c] = 1 << 29;
    }
#pragma unroll 1
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll 1
    for (int p = 0; p < kKs / 2; ++p) {
      const int aoff = (((p >> 1) ^ sw) << 2) + ((p & 1) << 1);
      float2 ap[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)
        asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];"
                     : "=f"(ap[r].x), "=f"(ap[r].y)
                     : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(A + 16 * r * kKs + aoff))));
      float4 bq[4];
#pragma unroll
      for (int m = 0; m < 4; ++m)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(bq[m].x), "=f"(bq[m].y), "=f"(bq[m].z), "=f"(bq[m].w)
                     : "r"(static_cast<uint32_t>(__cvta_generic_to_shared(B + p * 2 * kCols + 64 * m))));
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          if constexpr (FORM == 4) {
            const float2 s0 = __fadd2_rn(ap[r], make_float2(bq[m].x, bq[m].y));
            const float2 s1 = __fadd2_rn(ap[r], make_float2(bq[m].z, bq[m].w));
            acc[r][2 * m] = min3f(acc[r][2 * m], s0.x, s0.y);
            acc[r][2 * m + 1] = min3f(acc[r][2 * m + 1], s1.x, s1.y);
          } else if constexpr (FORM == 6) {
            acc[r][2 * m] = min3f(acc[r][2 * m], __fadd_rn(ap[r].x, bq[m].x), __fadd_rn(ap[r].y, bq[m].y));
            acc[r][2 * m + 1] =
                min3f(acc[r][2 * m + 1], __fadd_rn(ap[r].x, bq[m].z), __fadd_rn(ap[r].y, bq[m].w));
          } else if constexpr (FORM == 7) {
            const float2 s0 = __fadd2_rn(ap[r], make_float2(bq[m].x, bq[m].y));
            acc[r][2 * m] = min3f(acc[r][2 * m], s0.x, s0.y);
            acc[r][2 * m + 1] =
                min3f(acc[r][2 * m + 1], __fadd_rn(ap[r].x, bq[m].z), __fadd_rn(ap[r].y, bq[m].w));
          } else if constexpr (FORM == 8) {
            const int32_t a0 = __float_as_int(ap[r].x), a1 = __float_as_int(ap[r].y);
            int32_t s0, s1, s2;
            asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(s0) : "r"(a0), "r"(one), "r"(__float_as_int(bq[m].x)));
            asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(s1) : "r"(a1), "r"(one), "r"(__float_as_int(bq[m].y)));
            asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(s2) : "r"(a0), "r"(one), "r"(__float_as_int(bq[m].z)));
            iacc[r][2 * m] = __vimin3_s32(iacc[r][2 * m], s0, s1);
            iacc[r][2 * m + 1] = __vimin3_s32(iacc[r][2 * m + 1], s2, a1 + __float_as_int(bq[m].w));
          } else {
            const int32_t a0 = __float_as_int(ap[r].x), a1 = __float_as_int(ap[r].y);
            iacc[r][2 * m] = __vimin3_s32(iacc[r][2 * m], a0 + __float_as_int(bq[m].x), a1 + __float_as_int(bq[m].y));
            iacc[r][2 * m + 1] =
                __vimin3_s32(iacc[r][2 * m + 1], a0 + __float_as_int(bq[m].z), a1 + __float_as_int(bq[m].w));
          }
        }
    }
  }
  if constexpr (FORM == 4 || FORM == 6 || FORM == 7) {
    float s = 1e30f;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) s = fminf(s, acc[r][c]);
    static_cast<float *>(sinkv)[blockIdx.x * blockDim.x + threadIdx.x] = s;
  } else {
    int32_t s = 1 << 30;
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) s = min(s, iacc[r][c]);
    static_cast<int32_t *>(sinkv)[blockIdx.x * blockDim.x + threadIdx.x] = s;
  }
}

}  // namespace

extern "C" int apsp_ubench_minplus(int form, int64_t iters, int blocks, int threads, void *sink, void *stream,
                                   double *relax_per_s) {
  if (!sink || !relax_per_s || iters <= 0 || form < 0 || form > 9) return APSP_EINVAL;
  if (threads != 256) return APSP_EINVAL;  // the micro-tile layout is fixed
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (blocks <= 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
    blocks = 2 * sms;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return APSP_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return APSP_ECUDA;
  }
  auto launch = [&](int64_t its) {
    switch (form) {
      case 0: ubench_kstep<int32_t, 0><<<blocks, 256, 0, st>>>(its, (int32_t *)sink); break;
      case 1: ubench_kstep<float, 1><<<blocks, 256, 0, st>>>(its, (float *)sink); break;
      case 2: ubench_kstep<uint32_t, 2><<<blocks, 256, 0, st>>>(its, (uint32_t *)sink); break;
      case 3: ubench_kstep<int32_t, 3><<<blocks, 256, 0, st>>>(its, (int32_t *)sink); break;
      case 4: ubench_kpair<4><<<blocks, 256, 0, st>>>(its, sink); break;
      case 5: ubench_kpair<5><<<blocks, 256, 0, st>>>(its, sink); break;
      case 6: ubench_kpair<6><<<blocks, 256, 0, st>>>(its, sink); break;
      case 7: ubench_kpair<7><<<blocks, 256, 0, st>>>(its, sink); break;
      case 8: ubench_kpair<8><<<blocks, 256, 0, st>>>(its, sink); break;
      case 9: ubench_s16x2_narrow<<<blocks, 256, 0, st>>>(its, (uint32_t *)sink); break;
    }
  };
  launch(iters / 8 + 1);  // warm-up (clocks, instruction cache)
  cudaEventRecord(e0, st);
  launch(iters);
  cudaEventRecord(e1, st);
  int rc = APSP_OK;
  float ms = 0.f;
  if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
      cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
    rc = APSP_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != APSP_OK) return rc;
  // relaxations per thread per sweep of the 32-k slice (int16x2: two per
  // lane; form 9 holds 32 lanes per thread, the others 64)
  const double per_sweep = (form == 2 ? 2.0 : 1.0) * 64.0 * kKs;
  *relax_per_s = (double)blocks * 256.0 * per_sweep * (double)iters / (ms * 1e-3);
  return APSP_OK;
}
