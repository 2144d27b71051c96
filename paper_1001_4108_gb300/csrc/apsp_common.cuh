// Shared device-side definitions of libapsp: value conventions, the
// relaxation w_ij <- min(w_ij, w_ik + w_kj) of Fig. 1 for each element type,
// and the inline-PTX helpers (mbarrier, TMA) of the staged phase-3 kernel.
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace apsp {

// Error codes a kernel can leave in the device error word.
enum DeviceError : int {
  kDevOk = 0,
  kDevTimeoutTma = 1,  // an mbarrier wait for a TMA copy gave up
};

// Longest a bounded device wait spins before giving up (nanoseconds).
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------------------
// Element types.  Each storage type T has a compute type C used in shared
// memory and registers, the "infinity" of its input convention, the
// relaxation, and the output finish (clamp) applied in the last stage.
// ---------------------------------------------------------------------------
template <typename T> struct Arith;

// int32: infinity = 2^29.  All entries stay <= 2^29 (they only decrease), so
// the sum of two entries is <= 2^30 and never overflows; any value >= 2^28 is
// "no path" under the documented weight bound and is written back as 2^29.
template <> struct Arith<int32_t> {
  using C = int32_t;
  static constexpr int32_t kInfHost = 1 << 29;
  __device__ __forceinline__ static C inf() { return 1 << 29; }
  __device__ __forceinline__ static C load(int32_t v) { return v; }
  __device__ __forceinline__ static C relax(C acc, C a, C b) {
    return __viaddmin_s32(a, b, acc);  // min(a + b, acc) as one DPX operation
  }
  __device__ __forceinline__ static int32_t finish(C v) { return v >= (1 << 28) ? (1 << 29) : v; }
};

// fp32: infinity = +inf, exact under + and min; a + b is rounded once, the
// minimum is exact, so the result does not depend on the order of the k's.
template <> struct Arith<float> {
  using C = float;
  __device__ __forceinline__ static C inf() { return __int_as_float(0x7f800000); }
  __device__ __forceinline__ static C load(float v) { return v; }
  __device__ __forceinline__ static C relax(C acc, C a, C b) { return fminf(acc, __fadd_rn(a, b)); }
  __device__ __forceinline__ static float finish(C v) { return v; }
};

// int16 (scalar kernels): computed in int32, infinity = 16383.  With
// non-negative weights and (n-1)*Wmax < 16383 entries stay in [0, 16383],
// sums fit easily and unreachable pairs end at exactly 16383.
template <> struct Arith<int16_t> {
  using C = int32_t;
  __device__ __forceinline__ static C inf() { return 16383; }
  __device__ __forceinline__ static C load(int16_t v) { return (C)v; }
  __device__ __forceinline__ static C relax(C acc, C a, C b) { return __viaddmin_s32(a, b, acc); }
  __device__ __forceinline__ static int16_t finish(C v) { return (int16_t)v; }
};

// ---------------------------------------------------------------------------
// PTX helpers (sm_90+ forms, valid on sm_103a).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// A shared-memory word read the compiler cannot hoist or merge: values kept
// in shared memory across a long loop instead of in registers.
__device__ __forceinline__ int lds_volatile(const int *p) {
  int v;
  asm volatile("ld.shared.b32 %0, [%1];" : "=r"(v) : "r"(smem_u32(p)) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the given phase of an mbarrier; gives up after limit_ns and
// returns false instead of hanging.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// Release of the stages of a TMA ring without a CTA barrier per slice.
// Every warp, once done with the slice in stage st, counts itself in; the
// last of the CTA's warps refills the stage with the slice STAGES further
// on.  So warps wait only for data, never for each other, and drift apart by
// less than the ring's depth.  (A CTA barrier per slice instead left each
// warp waiting for the slowest, and the SM's other CTA did not fill those
// waits.  Measured on the phase-3 kernels, together with dropping the CTA
// barrier after the last slice where the kernel allows it: int32 7 %,
// int16x2 4 %, fp32 1.2 % faster.)
// Lives in shared memory; one thread initialises it before a CTA barrier.
template <int STAGES>
struct RingCtl {
  int issued;        // slices issued so far; they go out in slice order
  int abort;         // a wait gave up: no further refills
  int rel[STAGES];   // warps done with the slice now in each stage
};

template <int STAGES>
__device__ __forceinline__ void ring_ctl_init(RingCtl<STAGES> *c, int issued) {
  c->issued = issued;
  c->abort = 0;
#pragma unroll
  for (int s = 0; s < STAGES; ++s) c->rel[s] = 0;
}

// Called by every thread of the CTA after its last read of stage st.
// refill() issues the next slice into the stage (one thread runs it).
template <int STAGES, int NWARP, typename F>
__device__ __forceinline__ void ring_release(RingCtl<STAGES> *c, int st, bool timed_out, F &&refill) {
  asm volatile("" ::: "memory");
  __syncwarp();  // the whole warp is done reading the stage
  if ((threadIdx.x & 31) == 0) {
    if (timed_out) {
      atomicOr(&c->abort, 1);
      __threadfence_block();  // seen by whichever warp counts itself in last
    }
    if (atomicAdd(&c->rel[st], 1) == NWARP - 1) {
      atomicExch(&c->rel[st], 0);
      if (atomicOr(&c->abort, 0) == 0) {
        refill();
        atomicAdd(&c->issued, 1);
      }
    }
  }
}

// After a wait gave up (one thread: after a CTA barrier, or lane 0 of a warp
// that leaves on its own): records the error and waits (bounded again) for
// the copies that can still be in flight -- the last slice issued into each
// stage -- so that none lands in shared memory after the CTA has left.  (The
// CTA's shared memory lives until its last warp leaves, and a warp leaves
// only after waiting for every slice it read or draining like this.)
template <int STAGES>
__device__ __forceinline__ void ring_drain(RingCtl<STAGES> *c, uint64_t *full, int *err) {
  atomicCAS(err, 0, (int)kDevTimeoutTma);
  const int ni = *reinterpret_cast<volatile int *>(&c->issued);
  for (int g = ni > STAGES ? ni - STAGES : 0; g < ni; ++g) mbar_wait_bounded(&full[g % STAGES], (g / STAGES) & 1);
}

// 2-D tiled TMA load global -> shared, completion counted on an mbarrier.
// (x, y) = (column, row) of the box origin; x * sizeof(elem) % 16 == 0.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Index of a pivot-excluding tile: tiles b (the pivot block) is skipped.
// Programmatic dependent launch.  The stage kernels are launched with
// cudaLaunchAttributeProgrammaticStreamSerialization, so one may be scheduled
// while the kernel before it on the stream is still finishing (its launch and
// prologue overlap that kernel's tail).  Each calls this before its first
// access to the matrix or the panel workspace: it returns once the prior grid
// has completed and its writes are visible.  Without that attribute it
// returns at once.  APSP_PDL=0 builds both sides without it.
#ifndef APSP_PDL
#define APSP_PDL 1
#endif
__device__ __forceinline__ void wait_prior_grid() {
#if APSP_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");
#endif
}

__device__ __forceinline__ int skip_pivot(int t, int b) { return t < b ? t : t + 1; }

}  // namespace apsp
