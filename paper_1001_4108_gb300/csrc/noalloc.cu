// apsp_fw_f32_noalloc: the fp32 solve with its scratch in a file-scope device
// array instead of memory obtained from cudaMalloc.
//
// Some callers cannot allocate device memory on the solve path: a plugin
// inside a host framework that owns every byte of device memory through its
// own pool and forbids raw cudaMalloc; a latency-critical service that cannot
// absorb cudaMalloc / cudaFree (cudaFree synchronizes the whole device, and
// either call can fail in the middle of a request under a fixed memory
// budget).  This entry point gives them the packed fp32 kernels without any
// allocation: the k-pair interleaved row panel that phase 2 writes and
// phase 3 reads lives in `g_static_panel` below, which every GPU that loads
// the library holds until the process exits.
#include <mutex>

#include "../../include/apsp.h"
#include "apsp_internal.h"

namespace {

// Largest n served: the interleaved panel takes s * ceil(n/s) * s * 4 bytes,
// 8 MiB at n = 16384 (s = 128).
constexpr int64_t kMaxN = 16384;
constexpr size_t kPanelFloats = (size_t)128 * kMaxN;

// In host code this name is a host-side stand-in, not a device address; the
// kernels get the address returned by cudaGetSymbolAddress for the device.
static __device__ __align__(256) float g_static_panel[kPanelFloats];

constexpr int kMaxDev = 64;
std::mutex g_mu;
float *g_panel_ptr[kMaxDev];

// Once per device, with that device current: the device address of the array.
float *panel_for_current_device(int *status) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    *status = APSP_ECUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_panel_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_panel) != cudaSuccess || !p) {
      *status = APSP_ECUDA;
      return nullptr;
    }
    g_panel_ptr[dev] = static_cast<float *>(p);
  }
  *status = APSP_OK;
  return g_panel_ptr[dev];
}

}  // namespace

extern "C" int apsp_fw_f32_noalloc(void *dist, int64_t n, int64_t ld, void *stream) {
  if (n < 0 || ld < n) return APSP_EINVAL;
  if (n > kMaxN) return APSP_EUNSUPPORTED;
  if (n > 0 && !dist) return APSP_EINVAL;
  if (n == 0) return APSP_OK;
  int st = APSP_OK;
  float *panel = panel_for_current_device(&st);
  if (st != APSP_OK) return st;
  int *err = nullptr;
  st = apsp::error_word(&err);
  if (st != APSP_OK) return st;

  apsp::RunArgs a{};
  a.d = dist;
  a.n = n;
  a.ld = ld;
  a.S = apsp::default_kblock(n, APSP_F32);
  a.flags = 0;
  a.stream = static_cast<cudaStream_t>(stream);
  a.err = err;
  a.tma_ok = reinterpret_cast<uintptr_t>(dist) % 16 == 0 && ((size_t)ld * sizeof(float)) % 16 == 0;
  a.ws = panel;
  a.ws_bytes = kPanelFloats * sizeof(float);
  // One panel buffer always fits (s * ceil(n/s) * s floats <= 128 * 16384),
  // so the solve takes the plain schedule on the static array; whenever the
  // layout allows the packed kernels they must use it (the run refuses
  // rather than fall back to the unpacked kernels without telling).
  if (apsp::interleaved_panel_bytes(n, a.S) > a.ws_bytes) return APSP_EUNSUPPORTED;
  a.require_ws = true;
  return apsp::run_f32(a);
}
