// Host-side interface between the C-ABI translation unit (api.cu) and the
// per-element-type translation units (fw_i32.cu, fw_f32.cu, fw_i16.cu).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace apsp {

struct RunArgs {
  void *d;            // device matrix
  int64_t n, ld;      // vertices, leading dimension (elements)
  int S;              // tile side = k-block depth (64 or 128)
  int flags;          // APSP_FLAG_*
  void **events;      // optional per-phase events (kEventsPerStage per stage) or nullptr
  int64_t n_events;
  cudaStream_t stream;
  int *err;           // device error word
  bool tma_ok;        // layout allows the TMA-staged phase 3
  void *ws;           // device workspace (256-byte aligned) or nullptr
  size_t ws_bytes;
  // Lookahead schedule: a second stream of higher priority (nullptr = off)
  // and two events for the fork and join between it and `stream`.
  cudaStream_t side;
  cudaEvent_t fork, join;
  int side_prio;      // launch priority of the side-stream kernels
  // Optional path bookkeeping: via[i * via_ld + j] = stage of the last strict
  // improvement of d_ij (nullptr = off).
  int16_t *via;
  int64_t via_ld;
  // Optional routing of the C tiles of phase 3 (host entry point): stage 0
  // reads them from first_src and the last stage writes them to last_dst,
  // both device-accessible host memory with their own leading dimensions
  // (nullptr = the matrix).  Needs whole tiles and the TMA kernels; a run
  // that cannot honor it returns APSP_EUNSUPPORTED before enqueueing work.
  const void *first_src;
  int64_t first_src_ld;
  void *last_dst;
  int64_t last_dst_ld;
  // fp32: the packed phase-3 kernels must run on `ws` whenever tma_ok holds
  // and there are two stages or more; otherwise the run returns
  // APSP_EUNSUPPORTED before enqueueing work.
  bool require_ws;
};

// One-launch schedule for small matrices (dataflow.cu, APSP_FLAG_ONE_LAUNCH):
// s = 64 and a stage count in [kDataflowMinRounds, kDataflowMaxRounds].  Its
// per-tile flags (dataflow_flag_bytes) live at the start of the workspace.
// run_dataflow returns an apsp_status.
constexpr int kDataflowMinRounds = 2;
constexpr int kDataflowMaxRounds = 32;
size_t dataflow_flag_bytes(int R);
int run_dataflow(const RunArgs &a, int dtype, int *flags);

// Events a traced solve records per stage (apsp_options.events).
constexpr int kEventsPerStage = 5;
// Smallest tile-grid side R for which the lookahead schedule is used.
constexpr int kLookaheadMinRounds = 3;

// Largest R for which the s = 64 panel and cross launches are cut into strips
// (fw_strip).  While the bulk launch of a stage ((R-1)^2 tiles) fills only a
// wave or two of the GPU, the stage waits on the panel/cross chain, and four
// times as many CTAs per launch shorten it; beyond, the bulk launch bounds the
// stage and the strips only take SM time from it.  Solve times with strips
// against without, measured on GB300:
//   R      24    32    40    48    56    64
//   fp32  -29%  -23%  -13%   -2%   +4%   +8%
//   int32 -12%  -18%   +8%  +11%   +6%   +5%
// APSP_STRIP_MAX_ROUNDS (a build define) sets both limits, for such sweeps.
#ifdef APSP_STRIP_MAX_ROUNDS
constexpr int kStripMaxRoundsF32 = APSP_STRIP_MAX_ROUNDS, kStripMaxRoundsI32 = APSP_STRIP_MAX_ROUNDS;
#else
constexpr int kStripMaxRoundsF32 = 48, kStripMaxRoundsI32 = 32;
#endif
// Whether a solve with tile side S and R stages cuts its panel (and cross)
// tiles into strips; int16 keeps its packed kernels.
inline bool uses_strips(int S, int R, bool f32, bool i16) {
  return S == 64 && !i16 && R >= 2 && R <= (f32 ? kStripMaxRoundsF32 : kStripMaxRoundsI32);
}

// Workspace bytes of the packed int16x2 phase 3 (replicated column panel:
// n_p rows x s words).
inline size_t replicated_panel_bytes(int64_t n, int S) {
  const int64_t np = (n + S - 1) / S * S;
  return (size_t)np * (size_t)S * sizeof(uint32_t);
}

// Workspace bytes of the packed fp32 phase 3 (interleaved row panel).
inline size_t interleaved_panel_bytes(int64_t n, int S) {
  const int64_t np = (n + S - 1) / S * S;
  return (size_t)S * (size_t)np * sizeof(float);
}

// One graph of a batch (device matrix, leading dimension, vertices).
struct BatchDesc {
  void *d;
  int64_t ld;
  int64_t n;
};
// Largest n the one-CTA-per-graph batched kernel takes; larger graphs of a
// batch go through the multi-CTA path.
constexpr int64_t kBatchCtaMaxN = 512;
// Solves graphs (all n <= kBatchCtaMaxN, sorted largest first) with the
// persistent batched kernel.  Returns an apsp_status.
int run_batched_small(const BatchDesc *host_descs, int count, int dtype, cudaStream_t st, int dev);

// Autotuned choices (defaults until apsp_autotune / apsp_tuning_load).
// Batched kernel shapes: 0 = (s 32, 2x2), 1 = (s 32, 4x4), 2 = (s 64, 4x4),
// 3 = (s 128, 4x4).
constexpr int kBatchVariants = 4;
int tuned_batch_variant(int64_t n, int dtype);
int tuned_kblock(int64_t n, int dtype);
// match_single: graphs with n > 32 take the s = 64 shape, so that each result
// is bit-identical to apsp_fw's for that graph (s = 64 up to n = 512, and the
// same per-element operations in every kernel).
int run_batched_direct(const BatchDesc *host_descs, int count, int dtype, cudaStream_t st, void **dev_buf,
                       size_t *cap, bool match_single = false);
int time_batched_variant(const BatchDesc *dev_descs, int count, int *counter, int dtype, int variant,
                         cudaStream_t st, float *ms);

// Enqueue every stage of Fig. 2 for one matrix.  Returns an apsp_status.
int run_i32(const RunArgs &a);
int run_f32(const RunArgs &a);
int run_i16(const RunArgs &a);

// Checks and conversions around a solve (checks.cu); each returns an
// apsp_status.  validate_input and check_negcycle synchronize the stream.
int validate_input(const void *dist, int64_t n, int64_t ld, int dtype, cudaStream_t st, bool narrow);
int check_negcycle(void *dist, int64_t n, int64_t ld, int dtype, cudaStream_t st, int *neg);
int narrow_to_i16(const int32_t *src, int64_t n, int64_t ld, int16_t *dst, int64_t ld16, cudaStream_t st);
int widen_from_i16(const int16_t *src, int64_t ld16, int64_t n, int32_t *dst, int64_t ld, cudaStream_t st);

// Tile side the C ABI picks for (n, dtype) when none is requested.
int default_kblock(int64_t n, int dtype);
// Device address of the device error word of the current device (set-up once
// per device, no allocation).  Returns an apsp_status.
int error_word(int **err);

// cuTensorMapEncodeTiled from the driver, resolved once (nullptr if absent).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled_fn();

}  // namespace apsp
