// Roofline calibration for the min-plus relaxation (apsp_ubench_minplus).
//
// Each thread keeps the same 8 x 8 register micro-tile as the phase-3 kernel
// and applies acc[r][c] <- min(acc[r][c], a[r] + b[c]) with no memory traffic
// in the loop.  An empty asm statement marks a[] and b[] as rewritten every
// iteration, so the compiler can neither fold repeated minima nor hoist the
// additions, at no instruction cost.  The measured relaxations per second,
// divided by SMs x clock, give lanes per clock per SM for each form.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apsp.h"

namespace {

template <typename T> __device__ __forceinline__ void opaque(T &x);
template <> __device__ __forceinline__ void opaque<int32_t>(int32_t &x) { asm volatile("" : "+r"(x)); }
template <> __device__ __forceinline__ void opaque<uint32_t>(uint32_t &x) { asm volatile("" : "+r"(x)); }
template <> __device__ __forceinline__ void opaque<float>(float &x) { asm volatile("" : "+f"(x)); }

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

// form 0/3: int32, form 1: fp32, form 2: int16x2
template <typename T, int FORM>
__global__ void ubench_kernel(int64_t iters, T *sink) {
  T a[8], b[8], acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    a[r] = (T)(threadIdx.x + r);
    b[r] = (T)(blockIdx.x + 3 * r);
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = (T)(1 << 20);
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      opaque<T>(a[r]);
      opaque<T>(b[r]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if constexpr (FORM == 0) acc[r][c] = relax_dpx(acc[r][c], a[r], b[c]);
        if constexpr (FORM == 1) acc[r][c] = relax_f32(acc[r][c], a[r], b[c]);
        if constexpr (FORM == 2) acc[r][c] = relax_s16x2(acc[r][c], a[r], b[c]);
        if constexpr (FORM == 3) acc[r][c] = relax_addmin(acc[r][c], a[r], b[c]);
      }
  }
  T s = acc[0][0];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s = (r + c) ? (acc[r][c] < s ? acc[r][c] : s) : s;
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// form 4: fp32 with packed f32x2 additions (two k's at once) and a three-input
// minimum: acc <- min(acc, a0 + b0, a1 + b1), 2 relaxations per 2 instructions.
__global__ void ubench_f32x2(int64_t iters, float *sink) {
  float a0[8], a1[8], b0[8], b1[8], acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    a0[r] = threadIdx.x + r;
    a1[r] = threadIdx.x - r;
    b0[r] = blockIdx.x + 3 * r;
    b1[r] = blockIdx.x - 3 * r;
  }
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 1e20f;
  for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      opaque<float>(a0[r]);
      opaque<float>(a1[r]);
      opaque<float>(b0[r]);
      opaque<float>(b1[r]);
    }
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint64_t av, bv, sv;
        asm("mov.b64 %0, {%1, %2};" : "=l"(av) : "f"(a0[r]), "f"(a1[r]));
        asm("mov.b64 %0, {%1, %2};" : "=l"(bv) : "f"(b0[c]), "f"(b1[c]));
        asm("add.rn.f32x2 %0, %1, %2;" : "=l"(sv) : "l"(av), "l"(bv));
        float s0, s1;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(s0), "=f"(s1) : "l"(sv));
        asm("min.f32 %0, %1, %2, %3;" : "=f"(acc[r][c]) : "f"(acc[r][c]), "f"(s0), "f"(s1));
      }
  }
  float s = 1e30f;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fminf(s, acc[r][c]);
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" int apsp_ubench_minplus(int form, int64_t iters, int blocks, int threads, void *sink, void *stream,
                                   double *relax_per_s) {
  if (!sink || !relax_per_s || iters <= 0 || threads <= 0 || threads > 1024 || form < 0 || form > 4)
    return APSP_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (blocks <= 0) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return APSP_ECUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return APSP_ECUDA;
    blocks = 4 * sms;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return APSP_ECUDA;
  auto launch = [&](int64_t its) {
    switch (form) {
      case 0: ubench_kernel<int32_t, 0><<<blocks, threads, 0, st>>>(its, (int32_t *)sink); break;
      case 1: ubench_kernel<float, 1><<<blocks, threads, 0, st>>>(its, (float *)sink); break;
      case 2: ubench_kernel<uint32_t, 2><<<blocks, threads, 0, st>>>(its, (uint32_t *)sink); break;
      case 3: ubench_kernel<int32_t, 3><<<blocks, threads, 0, st>>>(its, (int32_t *)sink); break;
      case 4: ubench_f32x2<<<blocks, threads, 0, st>>>(its, (float *)sink); break;
    }
  };
  launch(iters / 8 + 1);  // warm-up (clocks, instruction cache)
  cudaEventRecord(e0, st);
  launch(iters);
  cudaEventRecord(e1, st);
  int rc = APSP_OK;
  float ms = 0.f;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = APSP_ECUDA;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != APSP_OK) return rc;
  const double per_lane = (form == 2 || form == 4) ? 128.0 : 64.0;  // relaxations per iteration per thread
  *relax_per_s = (double)blocks * threads * per_lane * (double)iters / (ms * 1e-3);
  return APSP_OK;
}
