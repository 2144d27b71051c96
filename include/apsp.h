/*
 * apsp.h -- C ABI of libapsp, a GB300 (sm_103a) implementation of the blocked
 * Floyd-Warshall all-pairs shortest-paths method of Lund & Smith, "A
 * Multi-Stage CUDA Kernel for Floyd-Warshall".
 *
 * Problem (Sec. 3.1): a directed graph on n vertices is given by its n x n
 * weight matrix W: w_ij is the weight of edge (v_i, v_j), "infinity" when the
 * edge is absent, w_ii = 0, and no cycle has negative total weight.  The
 * result d_ij (length of a shortest path from v_i to v_j) overwrites W in
 * place, exactly as Fig. 1 leaves d^(n) in the incidence matrix.
 *
 * Method (Sec. 3.2, Fig. 2): the matrix is cut into s x s tiles; for every
 * k-block b the "independent" diagonal tile is closed first (phase 1), then
 * the "singly dependent" tiles of row b and column b (phase 2), then all other
 * "doubly dependent" tiles, whose relaxations may run in any order (phase 3).
 *
 * Matrix layout for every entry point: row-major, leading dimension ld >= n
 * (in elements); only the n x n leading block is read or written, columns
 * n..ld-1 of each row are never touched.
 *
 * Value conventions
 *   APSP_I32  int32_t.  Absent edge / unreachable pair = APSP_INF_I32 (2^29).
 *             Inputs must satisfy w_ij <= 2^29 and (n-1)*(Wmax+|Wmin|) < 2^28,
 *             where Wmax/Wmin range over the present edges; every output that
 *             is >= 2^28 is written as 2^29.  The result is exact.
 *   APSP_F32  float.  Absent edge / unreachable pair = +infinity.  Results
 *             are computed with fp32 additions and exact minima; they are
 *             bit-exact when all path sums are exactly representable.
 *   APSP_I16  int16_t.  Absent edge / unreachable pair = APSP_INF_I16 (16383).
 *             Requires non-negative weights with (n-1)*Wmax < 16383, so that no
 *             sum of two entries leaves int16 and every unreachable pair ends
 *             at exactly 16383; the result is exact.  Two adjacent columns are
 *             relaxed per 32-bit lane (packed int16x2).
 *
 * Errors: every entry point returns an apsp_status.  Argument errors are
 * reported synchronously and leave the matrix untouched.  Kernels are
 * stream-ordered; an error that happens on the device is reported by the
 * next call that synchronizes (APSP_ECUDA) or by apsp_device_error().
 * A negative cycle in the input is not an error the library can see in
 * general: the output is then unspecified (the paper excludes it).
 *
 * Threading: all entry points are reentrant for distinct matrices.
 */
#ifndef APSP_H
#define APSP_H

#include <stdint.h>

#if defined(__GNUC__)
#define APSP_API __attribute__((visibility("default")))
#else
#define APSP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define APSP_INF_I32 (1 << 29)
#define APSP_CLAMP_I32 (1 << 28)
#define APSP_INF_I16 16383

typedef enum apsp_dtype {
    APSP_I32 = 0,
    APSP_F32 = 1,
    APSP_I16 = 2
} apsp_dtype;

typedef enum apsp_status {
    APSP_OK = 0,
    APSP_EINVAL = 1,      /* bad argument (null pointer, n < 0, ld < n, ...)  */
    APSP_ENOMEM = 2,      /* an allocation failed                              */
    APSP_EUNSUPPORTED = 3,/* valid request the library cannot serve           */
    APSP_ECUDA = 4,       /* a CUDA runtime call failed                        */
    APSP_ETIMEOUT = 5,    /* a bounded device-side wait gave up                */
    APSP_EBUSY = 6,       /* resource in use (serving: no slot / memory)       */
    APSP_EPENDING = 7,    /* serving: result not ready yet                     */
    APSP_ENEGCYCLE = 8    /* negative cycle detected (only when asked)         */
} apsp_status;

/* Flags for apsp_options.flags. */
#define APSP_FLAG_NO_GRAPH   0x1  /* launch the round loop directly, no CUDA graph        */
#define APSP_FLAG_GENERIC    0x2  /* force the generic (non-TMA) phase-3 kernel           */
#define APSP_FLAG_REVERSE_K  0x4  /* phase 3 visits the k-block in reverse order.  The
                                     result must not change: the tasks of a doubly
                                     dependent tile may run in any order (Sec. 3.2).     */
#define APSP_FLAG_NEGCYCLE   0x8  /* after the solve, report APSP_ENEGCYCLE if some d_ii < 0
                                     (synchronizes the stream)                           */
#define APSP_FLAG_NO_WORKSPACE 0x10 /* use only kernels that need no device workspace
                                     (same results, slower for fp32)                     */
#define APSP_FLAG_NO_LOOKAHEAD 0x20 /* plain stage order: phases 1 and 2 of stage b+1 do
                                     not overlap phase 3 of stage b (same results)       */
#define APSP_FLAG_NARROW     0x80 /* APSP_I32 only: the caller states that every weight is
                                     >= 0 and (n-1)*Wmax < 16383 (APSP_FLAG_VALIDATE then
                                     checks exactly that); the matrix is copied to int16,
                                     solved by the packed int16x2 kernels (about twice the
                                     rate) and copied back, with absent = 2^29 in and out.
                                     Same results as the int32 path.  Uses library memory
                                     (n^2 x 2 bytes + int16 panels, per device and stream);
                                     APSP_EINVAL with a caller workspace or apsp_fw_paths. */
#define APSP_FLAG_ONE_LAUNCH 0x100 /* small matrices (s = 64, 2 to 32 stages): every
                                     stage in one cooperative launch, the tiles spread
                                     over the CTAs and ordered by per-tile flags in the
                                     workspace ((3 R^2 + R) x 4 bytes, R = stages; with a
                                     smaller caller workspace, or with GENERIC,
                                     REVERSE_K, NO_LOOKAHEAD, tracing or apsp_fw_paths,
                                     the multi-launch schedule runs).  Same results.
                                     Not faster than the default on GB300 (measured:
                                     n = 1024 fp32 333 vs 266 us); kept for study.  A
                                     flag wait that runs out (2 s) sets the device
                                     error word to 2 (apsp_device_error).              */
#define APSP_FLAG_VALIDATE   0x40 /* before solving, check the input against the value
                                     conventions above (one pass over the matrix, then a
                                     stream synchronize): int32 entries <= 2^29 and
                                     (n-1)(Wmax+|Wmin|) < 2^28; int16 entries in
                                     [0, 16383] and (n-1)Wmax < 16383; fp32 no NaN.
                                     APSP_EINVAL if violated.  This flag and
                                     APSP_FLAG_NEGCYCLE synchronize, so they are refused
                                     (APSP_EINVAL) while the stream is being captured.  */

typedef struct apsp_options {
    int32_t kblock;          /* k-block depth s (64 or 128); 0 = chosen from n and dtype */
    int32_t flags;           /* APSP_FLAG_* */
    /* Optional tracing: an array of cudaEvent_t (cast to void*) of length
       5 * rounds.  For stage r the library records events[5r] before phase 1,
       [5r+1] before phase 2, [5r+2] after phase 2, [5r+3] before and [5r+4]
       after the phase-3 launch on the call's stream.  With the lookahead
       schedule (apsp_config.lookahead) phases 1 and 2 of stage r > 0 run on an
       internal stream beside phase 3 of stage r-1, so events 5r..5r+2 are
       recorded there, and the phase-3 launch on the call's stream covers every
       tile except row and column r+1 (those run on the internal stream
       before phase 1 of stage r+1, untimed).  Tracing implies
       APSP_FLAG_NO_GRAPH.  NULL = off. */
    void **events;
    int64_t n_events;
    /* Optional device workspace of apsp_workspace_bytes(n, dtype, kblock)
       bytes (at least one panel buffer, half of that from 3 stages on: then
       the plain schedule runs), 256-byte aligned, owned by the caller and used
       only between the enqueue and the completion of this call's work on its
       stream; smaller: APSP_EINVAL.
       NULL = the library uses a buffer of its own, one per (device, stream),
       allocated on first use (not while the stream is being captured). */
    void *workspace;
    int64_t workspace_bytes;
} apsp_options;

/* Kernel configuration the library picks for (n, dtype); see apsp_options. */
typedef struct apsp_config {
    int32_t kblock;          /* s: tile side and k-block depth                     */
    int32_t rounds;          /* ceil(n / s): stages of Fig. 2                       */
    int32_t phase3_tma;      /* 1 if the TMA-staged phase-3 kernel is used          */
    int32_t phase3_threads;  /* threads per phase-3 CTA                             */
    int64_t phase3_relax_per_round; /* relaxations phase 3 performs in a full round */
    int32_t lookahead;       /* 1 if a call without flags uses the lookahead schedule
                                (stages >= 3, TMA-staged kernels, library workspace) */
    int32_t strips;          /* 1 if a call without flags on 16-byte aligned rows cuts
                                each 64 x 64 tile of its phase-2 launches (and of the
                                lookahead's cross launches) into four one-CTA strips:
                                s = 64, fp32 up to 48 stages, int32 up to 32 */
} apsp_config;

/* Status name, e.g. "APSP_EINVAL".  Never NULL. */
APSP_API const char *apsp_status_str(int status);

/* Library version as major*10000 + minor*100 + patch. */
APSP_API int apsp_version(void);

/*
 * All-pairs shortest paths in place (Fig. 2, blocked Floyd-Warshall).
 *   dist   device pointer to the n x n matrix (row-major, leading dim ld);
 *          owned by the caller; overwritten with the distances.
 *   n      vertices (0 is a no-op).
 *   ld     leading dimension in elements, ld >= n.
 *   dtype  APSP_I32 / APSP_F32 / APSP_I16.
 *   stream cudaStream_t (cast to void*); NULL = legacy default stream.
 * Stream-ordered: returns after the work is enqueued.  The fast phase-3 path
 * needs dist 16-byte aligned and ld*sizeof(element) a multiple of 16; other
 * layouts run a generic kernel (same results, slower).
 * Returns APSP_EINVAL on a bad argument, APSP_ECUDA if a launch fails.
 */
APSP_API int apsp_fw(void *dist, int64_t n, int64_t ld, int dtype, void *stream);

/*
 * Many independent graphs in one call (e.g. thousands of small graphs).
 *   dists  host array of `count` device pointers (matrices in place);
 *   ns, lds host arrays of vertex counts and leading dimensions;
 *   dtype  one element type for all graphs.
 * The arrays are read before the call returns (the caller keeps ownership).
 * Graphs with n <= 512 are solved by one persistent launch in which each CTA
 * takes a graph (largest first) and runs all stages of Fig. 2 for it; larger
 * graphs use the apsp_fw path.  Solving the same batch (same matrices and
 * stream) again replays a CUDA graph of that launch.  Not allowed while the
 * stream is being captured (APSP_EUNSUPPORTED).  Results equal apsp_fw's for
 * integers; for fp32 they agree within the rounding of the additions.
 * Returns the first argument error (before any work) or APSP_ECUDA.
 */
APSP_API int apsp_fw_batched(void *const *dists, const int64_t *ns, const int64_t *lds, int64_t count, int dtype,
                             void *stream);

/* apsp_fw with options (NULL = defaults).  See apsp_options. */
APSP_API int apsp_fw_ex(void *dist, int64_t n, int64_t ld, int dtype, const apsp_options *opt,
               void *stream);

/*
 * apsp_fw on a matrix in HOST memory (pinned or pageable).  The library copies
 * it to a device buffer it owns (kept for reuse, one per device), solves in
 * place there and copies the result back.  Returns when the result is in
 * host_dist (synchronizes the stream).
 */
APSP_API int apsp_fw_host(void *host_dist, int64_t n, int64_t ld, int dtype, void *stream);

/*
 * Shortest paths, not only their lengths (the paper computes distances only,
 * Sec. 3.1; this is the path-reconstruction extension).
 *
 * apsp_fw_paths: apsp_fw_ex plus a stage record.  via (device, int16,
 * row-major, leading dimension via_ld >= n elements, owned by the caller,
 * written in full) receives, for every pair, the stage b (k-block b of
 * Fig. 2) whose relaxations last strictly lowered d_ij, or -1 if d_ij kept its
 * input value.  Every phase kernel compares the values it computes with the
 * ones they replace; distances are bit-identical to apsp_fw_ex.  The stage
 * numbers refer to the k-block depth of the solve (apsp_config.kblock for
 * the same n, dtype and options.kblock).  APSP_EUNSUPPORTED if the number of
 * stages exceeds 32767; other errors as apsp_fw_ex.
 *
 * apsp_path: one path i -> j from HOST copies of the solved matrix and of
 * via (same layouts and dtype as the solve; kblock = that solve's k-block
 * depth).  Writes the vertices i, ..., j to path (cap entries) and their
 * number to *len: 1 for i == j, 0 if j is unreachable from i.  Block b of a
 * pair (u, v) holds a vertex k with d_uk + d_kv = d_uv (integers: exactly,
 * since the last improvement used values that no later stage lowered;
 * fp32: the k whose rounded sum is nearest d_uv); the path is the edge
 * u -> v for -1, else path(u, k) + path(k, v).  APSP_ENOMEM if cap is too
 * small (*len then holds the length needed), APSP_EINVAL for bad arguments or
 * a record that does not match the matrix.
 */
APSP_API int apsp_fw_paths(void *dist, int16_t *via, int64_t n, int64_t ld, int64_t via_ld, int dtype,
                           const apsp_options *opt, void *stream);
APSP_API int apsp_path(const void *dist, const int16_t *via, int64_t n, int64_t ld, int64_t via_ld, int dtype,
                       int32_t kblock, int64_t i, int64_t j, int64_t *path, int64_t cap, int64_t *len);

/*
 * Device workspace (bytes) a solve of this size uses; 0 if none.  fp32 solves
 * keep a k-pair-interleaved copy of the current pivot row panel there, int16
 * solves a copy of the current pivot column panel with every entry duplicated
 * into both halves of a 32-bit word; both are s * ceil(n/s) * s * 4 bytes
 * (8 MiB at n = 16384, s = 128), written by phase 2 and read by phase 3.
 * From 3 stages on, two such buffers (the lookahead schedule writes the next
 * stage's copy while phase 3 reads the current one); a workspace holding one
 * buffer runs the plain schedule.  Without a workspace the same results come
 * from slower phase-3 kernels.
 */
APSP_API int64_t apsp_workspace_bytes(int64_t n, int dtype, int32_t kblock);

/*
 * apsp_fw for APSP_F32 that allocates nothing (the paper has no counterpart:
 * this serves callers that may not allocate device memory on the solve path,
 * e.g. a plugin whose host framework owns all device memory through its own
 * pool, or a latency-critical service that cannot absorb cudaMalloc/cudaFree,
 * which can fail mid-request and, for cudaFree, synchronize the device).
 *   dist, n, ld, stream  as in apsp_fw (fp32 matrix, in place; the caller
 *                        still owns and passes the matrix).
 * The scratch the packed phase 3 needs (the interleaved row panel) lives in a
 * static device array of the library, 8 MiB, held by every GPU that loads the
 * library until the process exits.  Limit: n <= 16384; larger n returns
 * APSP_EUNSUPPORTED before any device work.  With dist 16-byte aligned, ld * 4
 * a multiple of 16 and n above one tile, the solve always runs the packed
 * kernels on the array (if they cannot run, the call returns
 * APSP_EUNSUPPORTED before any device work); other layouts run the unpacked
 * kernels, which need no scratch.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  All calls share the one array and each
 * solve rewrites every part of it that it reads, so nothing needs clearing;
 * calls whose work overlaps on the GPU (e.g. on two streams at once) race on
 * it and must be serialized by the caller.  Launches kernels directly (no
 * library-owned graph, stream or workspace).  Stream-ordered like apsp_fw.
 */
APSP_API int apsp_fw_f32_noalloc(void *dist, int64_t n, int64_t ld, void *stream);

/*
 * Autotuner (the paper has none; in the spirit of the per-architecture code
 * generator it cites).  Times, on this GPU and for one element type:
 *   - the batched kernel shapes (tile side / register block per thread:
 *     32/2x2, 32/4x4, 64/4x4, 128/4x4) on synthetic batches for n buckets
 *     <= 32, 64, 128, 256, 512, keeping the fastest shape per bucket, then a
 *     few whole-batch assignments on a mixed batch;
 *   - the single-graph k-block depth (64 vs 128) at n = 1024 ... 6144,
 *     keeping the smallest n from which 128 stays faster.
 * The choices replace the built-in defaults for later calls in this process
 * (apsp_fw with kblock 0, apsp_fw_batched).  Allocates and frees its own test
 * matrices; synchronizes the stream; takes seconds.  If report != NULL, a JSON
 * summary of the timings is written there (truncated to report_len - 1 chars).
 */
APSP_API int apsp_autotune(int dtype, void *stream, char *report, int64_t report_len);

/* Save / load the tuning table (all element types) as a small text file.
   Load validates every entry and leaves the table unchanged on error
   (APSP_EINVAL). */
APSP_API int apsp_tuning_save(const char *path);
APSP_API int apsp_tuning_load(const char *path);

/*
 * Serving: a request loop with continuous batching.  apsp_submit copies the
 * request's host matrix and queues it; a scheduler thread of the server admits
 * queued requests oldest first while an in-flight slot is free and the
 * request's device footprint fits the HBM budget, uploads each admitted matrix
 * once and solves it on the device (requests with n <= 512 share one batched
 * launch, one CTA per graph, when at least 8 of one element type are admitted
 * together; the others run on their own streams, spread over all SMs, so
 * requests overlap on the GPU), copies the result back and releases the
 * device memory.  apsp_poll / apsp_wait deliver a finished result into the
 * caller's buffer and retire the ticket.  A result is the same whether the
 * request was solved alone or among others: integer results are exact, and
 * an fp32 request gets the same per-element operations in the same stage
 * order from either kernel (tile side 64 up to n = 512).  Latency is measured
 * from submit to the result being in host memory.
 */
typedef struct apsp_server apsp_server;  /* opaque, owned by the library */

typedef struct apsp_server_config {
    int32_t device;            /* CUDA device ordinal                                    */
    int32_t max_inflight;      /* requests on the GPU at once (slots), > 0               */
    int64_t hbm_budget_bytes;  /* device bytes the resident matrices may take, > 0       */
    int32_t streams;           /* streams for large requests (0 = 4)                     */
    int32_t flags;             /* reserved, 0                                            */
    int64_t max_n;             /* largest n accepted; sizes the per-stream workspaces     */
} apsp_server_config;

typedef struct apsp_stats {
    int64_t submitted, completed, failed, queued, inflight;
    int64_t bytes_resident;
    double p50_ms, p99_ms, mean_ms;  /* latency, submit -> result in host memory */
    double graphs_per_s;             /* completed / (last completion - first submit) */
} apsp_stats;

/* Creates a server (its scheduler thread, streams and workspaces). */
APSP_API int apsp_server_create(apsp_server **out, const apsp_server_config *cfg);

/* Queues one request; the matrix (host or device memory, row-major, leading
   dimension ld >= n) is copied before the call returns.  *ticket identifies
   it.  APSP_ENOMEM if the matrix alone exceeds the HBM budget,
   APSP_EUNSUPPORTED if n > max_n, APSP_EBUSY if the server is shutting down,
   APSP_ECUDA if copying from device memory fails. */
APSP_API int apsp_submit(apsp_server *srv, const void *host_dist, int64_t n, int64_t ld, int dtype, int flags,
                         uint64_t *ticket);

/* APSP_EPENDING while the request runs; otherwise delivers the distances
   into out_dist (host or device memory, leading dimension out_ld >= n;
   NULL = discard) and retires the ticket, returning APSP_OK or the request's
   error. */
APSP_API int apsp_poll(apsp_server *srv, uint64_t ticket, void *out_dist, int64_t out_ld);

/* apsp_poll that blocks up to timeout_us microseconds (< 0: no limit);
   APSP_ETIMEOUT if the request is still running then. */
APSP_API int apsp_wait(apsp_server *srv, uint64_t ticket, void *out_dist, int64_t out_ld, int64_t timeout_us);

/* Counters and latency percentiles; reset != 0 clears them afterwards. */
APSP_API int apsp_server_stats(apsp_server *srv, apsp_stats *out, int reset);

/* Stops admitting, waits for in-flight requests, fails queued ones, frees
   everything (undelivered results are dropped). */
APSP_API int apsp_server_destroy(apsp_server *srv);

/* Fills *cfg with the configuration apsp_fw would use (no device work). */
APSP_API int apsp_query_config(int64_t n, int dtype, int32_t kblock, apsp_config *cfg);

/*
 * Device error word: bounded device-side waits that give up set it instead of
 * hanging.  Returns 0 if clear, else the code of the first failure (and clears
 * it when reset != 0).  Synchronizes the device.
 */
APSP_API int apsp_device_error(int reset);

/*
 * Self-test of that failure path: enqueues one warp that waits on a barrier
 * phase nothing completes, gives up after limit_ns nanoseconds (1 ns .. 10 s)
 * and sets the device error word, exactly as a kernel's bounded wait does.
 * No fault and no hang: afterwards apsp_device_error() returns the timeout
 * code (1) and the context is usable.  APSP_EINVAL for a limit outside the
 * range.  (Not part of the paper: tests the library's own error plumbing.)
 */
APSP_API int apsp_selftest_wait(int64_t limit_ns, void *stream);

/*
 * Roofline calibration: runs the phase-3 inner loop of one instruction form on
 * every SM, with operands loaded from shared memory at every k step as in the
 * kernels (256 threads, 8 x 8 register micro-tile, a 32-k slice swept `iters`
 * times), and reports relaxations per second.
 *   form   0 int32 DPX add-min (one relaxation per instruction),
 *          1 fp32 add then min,
 *          2 int16x2 DPX add-min (two relaxations per instruction),
 *          3 int32 add then min as separate instructions,
 *          4 fp32 packed add.f32x2 + three-input min (two k's per pair),
 *          5 int32 two adds + three-input DPX min (two k's),
 *          6 fp32 two scalar adds + three-input min (two k's),
 *          7 fp32 forms 4 and 6 alternating by column,
 *          8 int32 additions three quarters as multiply-adds by a runtime 1
 *            (FMA pipe), one quarter as adds, + three-input DPX min,
 *          9 int16x2 DPX add-min on the int16x2 phase-3 kernel's own
 *            micro-tile (8 rows x 4 words, one 128-bit B load per k).
 *   iters  sweeps of the slice.
 *   blocks blocks to launch (<= 0: 2 per SM); threads must be 256.
 *   sink   device buffer of blocks*256 4-byte words (results are written so
 *          the work is not eliminated).
 *   relax_per_s  out: measured relaxations per second (host pointer).
 * Synchronizes the stream.
 */
APSP_API int apsp_ubench_minplus(int form, int64_t iters, int blocks, int threads, void *sink,
                        void *stream, double *relax_per_s);

#ifdef __cplusplus
}
#endif

#endif /* APSP_H */
