// Self-test of the failure path of the bounded device waits
// (apsp_selftest_wait): one warp waits on an mbarrier phase that nothing
// completes (no arrival, no copy), gives up after limit_ns and sets the
// device error word, as every kernel's TMA waits do.  A test can check the
// give-up path and that the context stays usable afterwards, without a fault.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/apsp.h"
#include "apsp_common.cuh"
#include "apsp_internal.h"

namespace {

__global__ void wait_never(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    apsp::mbar_init(&bar, 1);
    apsp::fence_mbar_init();
  }
  __syncthreads();
  const bool ok = apsp::mbar_wait_bounded(&bar, 0, limit_ns);
  if (__syncthreads_or(!ok) && threadIdx.x == 0) atomicCAS(err, 0, (int)apsp::kDevTimeoutTma);
}

}  // namespace

extern "C" int apsp_selftest_wait(int64_t limit_ns, void *stream) {
  if (limit_ns <= 0 || limit_ns > 10000000000ll) return APSP_EINVAL;
  int *err = nullptr;
  if (apsp::error_word(&err) != APSP_OK) return APSP_ECUDA;
  wait_never<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(err, (unsigned long long)limit_ns);
  return cudaPeekAtLastError() == cudaSuccess ? APSP_OK : APSP_ECUDA;
}
