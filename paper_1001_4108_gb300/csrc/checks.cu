// Checks and conversions around a solve: the input check of
// APSP_FLAG_VALIDATE, the negative-cycle report of APSP_FLAG_NEGCYCLE and the
// int32 <-> int16 copies of APSP_FLAG_NARROW.
#include <algorithm>
#include <climits>
#include <mutex>
#include <type_traits>

#include "../../include/apsp.h"
#include "apsp_internal.h"

// Input range of the validation pass: max finite entry, min entry, max
// entry, NaN seen.
static __device__ int g_apsp_range[4];

namespace apsp {

namespace {

template <typename T>
__global__ void diag_negative(const T *d, int64_t n, int64_t ld, int *flag) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (d[i * ld + i] < (T)0) atomicExch(flag, 1);
}

// One pass over the matrix: the largest entry below the dtype's infinity,
// the smallest entry, the largest entry overall and (fp32) whether a NaN
// occurs.  int16 entries are compared as int32.  Rows by blockIdx.y, columns
// by the threads of blockIdx.x (coalesced).
template <typename T>
__global__ void input_range(const T *d, int64_t n, int64_t ld, int inf, int *range) {
  int mx = INT_MIN, mn = INT_MAX, top = INT_MIN, nan = 0;
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const T v = d[i * ld + j];
      if constexpr (std::is_same<T, float>::value) {
        nan |= v != v;
      } else {
        const int x = (int)v;
        if (x < inf) mx = max(mx, x);
        mn = min(mn, x);
        top = max(top, x);
      }
    }
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    top = max(top, __shfl_xor_sync(0xffffffffu, top, o));
    nan |= __shfl_xor_sync(0xffffffffu, nan, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&range[0], mx);
    atomicMin(&range[1], mn);
    atomicMax(&range[2], top);
    if (nan) atomicExch(&range[3], 1);
  }
}

}  // namespace

// APSP_FLAG_VALIDATE: the value conventions of the header (synchronizes).
int validate_input(const void *dist, int64_t n, int64_t ld, int dtype, cudaStream_t st, bool narrow) {
  int *range = nullptr;
  if (cudaGetSymbolAddress(reinterpret_cast<void **>(&range), g_apsp_range) != cudaSuccess) return APSP_ECUDA;
  static std::mutex mu;  // one validation at a time uses the device words
  std::lock_guard<std::mutex> lk(mu);
  const int init[4] = {INT_MIN, INT_MAX, INT_MIN, 0};
  if (cudaMemcpyAsync(range, init, sizeof(init), cudaMemcpyHostToDevice, st) != cudaSuccess) return APSP_ECUDA;
  const dim3 grid((unsigned)std::min<int64_t>((n + 255) / 256, 4), (unsigned)std::min<int64_t>(n, 2048));
  if (dtype == APSP_I32)
    input_range<int32_t><<<grid, 256, 0, st>>>((const int32_t *)dist, n, ld, 1 << 29, range);
  if (dtype == APSP_F32) input_range<float><<<grid, 256, 0, st>>>((const float *)dist, n, ld, 0, range);
  if (dtype == APSP_I16) input_range<int16_t><<<grid, 256, 0, st>>>((const int16_t *)dist, n, ld, 16383, range);
  int h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, range, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return APSP_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return APSP_ECUDA;
  if (dtype == APSP_F32) return h[3] ? APSP_EINVAL : APSP_OK;
  const int64_t wmax = h[0] == INT_MIN ? 0 : std::max(h[0], 0), wneg = h[1] < 0 ? -(int64_t)h[1] : 0;
  if (dtype == APSP_I32 && narrow) {  // the int16 rules on int32 input
    if (h[2] > (1 << 29) || h[1] < 0) return APSP_EINVAL;
    return (n - 1) * wmax < 16383 ? APSP_OK : APSP_EINVAL;
  }
  if (dtype == APSP_I32) {
    if (h[2] > (1 << 29)) return APSP_EINVAL;  // above infinity
    return (n - 1) * (wmax + wneg) < (1 << 28) ? APSP_OK : APSP_EINVAL;
  }
  if (h[1] < 0) return APSP_EINVAL;  // int16: non-negative weights
  if (h[2] > 16383) return APSP_EINVAL;
  return (n - 1) * wmax < 16383 ? APSP_OK : APSP_EINVAL;
}

namespace {

// int32 <-> int16 copies of the narrowed solve (APSP_FLAG_NARROW).  Inputs
// obey the int16 bound, so every entry is either < 16383 or absent (2^29).
__global__ void narrow_i32(const int32_t *src, int64_t n, int64_t ld, int16_t *dst, int64_t ld16) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = src[i * ld + j];
      dst[i * ld16 + j] = (int16_t)(v >= 16383 ? 16383 : v);
    }
}
__global__ void widen_i16(const int16_t *src, int64_t ld16, int64_t n, int32_t *dst, int64_t ld) {
  for (int64_t i = blockIdx.y; i < n; i += gridDim.y)
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
      const int32_t v = src[i * ld16 + j];
      dst[i * ld + j] = v >= 16383 ? (1 << 29) : v;
    }
}
dim3 rows_grid(int64_t n) {
  return dim3((unsigned)std::min<int64_t>((n + 255) / 256, 4), (unsigned)std::min<int64_t>(n, 4096));
}

}  // namespace

int narrow_to_i16(const int32_t *src, int64_t n, int64_t ld, int16_t *dst, int64_t ld16, cudaStream_t st) {
  narrow_i32<<<rows_grid(n), 256, 0, st>>>(src, n, ld, dst, ld16);
  return cudaPeekAtLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

int widen_from_i16(const int16_t *src, int64_t ld16, int64_t n, int32_t *dst, int64_t ld, cudaStream_t st) {
  widen_i16<<<rows_grid(n), 256, 0, st>>>(src, ld16, n, dst, ld);
  return cudaPeekAtLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}

int check_negcycle(void *dist, int64_t n, int64_t ld, int dtype, cudaStream_t st, int *neg) {
  if (cudaMemsetAsync(neg, 0, sizeof(int), st) != cudaSuccess) return APSP_ECUDA;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 1024);
  if (dtype == APSP_I32) diag_negative<int32_t><<<blocks, 256, 0, st>>>((const int32_t *)dist, n, ld, neg);
  if (dtype == APSP_F32) diag_negative<float><<<blocks, 256, 0, st>>>((const float *)dist, n, ld, neg);
  if (dtype == APSP_I16) diag_negative<int16_t><<<blocks, 256, 0, st>>>((const int16_t *)dist, n, ld, neg);
  int h = 0;
  if (cudaMemcpyAsync(&h, neg, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return APSP_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return APSP_ECUDA;
  return h ? APSP_ENEGCYCLE : APSP_OK;
}

}  // namespace apsp
