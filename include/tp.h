/*
 * tp.h - C ABI of the partitioned tile-program library (libtp.so).
 *
 * The library runs the data-parallel hot path of "Fearless Concurrency on the
 * GPU" (cuTile Rust) on one GB300 (sm_103a): a grid of tile programs in which
 * each program owns a provably disjoint sub-tensor of a partitioned mutable
 * output (§3.4), computing element-wise maps (§2, Listing 1; §5.1) and tiled
 * GEMMs with a K loop (§3.6, Listing 6; §5.1), launched synchronously, as an
 * asynchronous stream pipeline, or by CUDA-graph replay (§3.2, Listings 2-3).
 *
 * Conventions shared by every entry point
 * - Every call returns a tp_status; no call aborts, exits or prints.
 *   tp_last_error_detail() gives a human-readable reason for the last failure
 *   on the calling thread.
 * - Pointers named "device" are CUDA device addresses (e.g. a torch tensor's
 *   data_ptr()); the library never frees memory it did not allocate.
 *   tp_tensor is a non-owning view (the borrow rows of Table 1, §3.3).
 * - Streams are cudaStream_t values passed as void* and are borrowed.
 * - Mutable outputs are passed as a tp_partition: an output tensor split into
 *   disjoint tiles (rank <= 3, §3.4). Inputs are read-only tp_tensor views and
 *   must not overlap the output's bytes (TP_ERR_ALIAS; §3.3, Appendix A).
 * - While an operation is in flight its partition is "busy" (the C analogue of
 *   the launch holding the tensor until the stream completes, §3.2 and §3.3):
 *   an operation on another stream that writes it or reads its bytes, or
 *   destroying or remapping it, returns TP_ERR_BUSY. Operations queued on the
 *   same stream run after it in stream order and may read or rewrite it: the
 *   analogue of chaining dependent work with `then` (§3.2). SYNC releases the
 *   hold before returning; ASYNC when tp_event_query reports completion or
 *   tp_event_wait returns; CAPTURE never marks it (the node has not run,
 *   §3.2) and graph replay holds the graph's partitions for its duration.
 * - Element strides are in elements. Dtype sizes: F32 4, BF16 2, F8E4M3 1.
 * - Nothing is allocated during graph capture (§3.2's rule that captured
 *   nodes are non-allocating); a call that would need to returns TP_ERR_CAPTURE.
 * - No call prints, except that with the environment variable TP_LOG set (to
 *   anything but "" or "0") every operation writes one trace line to stderr:
 *   entry point, outcome (done / enqueued / recorded / refused / aborted),
 *   mode, stream, the output's tiles and programs, and the status.
 */
#ifndef TP_H
#define TP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tp_status {
  TP_OK = 0,
  TP_ERR_INVALID = 1,     /* null or malformed argument / descriptor            */
  TP_ERR_RANK = 2,        /* mutable rank > 3, or rank mismatch                  */
  TP_ERR_ALIGN = 3,       /* pointer or stride misaligned for a TMA path         */
  TP_ERR_ALIAS = 4,       /* an input overlaps the output partition              */
  TP_ERR_BUSY = 5,        /* partition (or bytes an input reads) in flight       */
  TP_ERR_CAPTURE = 6,     /* not allowed while capturing a graph                 */
  TP_ERR_UNSUPPORTED = 7, /* valid request this build does not implement         */
  TP_ERR_CUDA = 8,        /* a CUDA runtime/driver call failed                   */
  TP_ERR_TIMEOUT = 9,     /* a device-side wait hit its iteration cap            */
  TP_ERR_SHAPE = 10,      /* operand shapes disagree                             */
  TP_ERR_RACE = 11        /* checked launch: a tile stored twice or off the map  */
} tp_status;

typedef enum tp_dtype {
  TP_F32 = 0,
  TP_BF16 = 1,
  TP_F8E4M3 = 2,
  TP_F64 = 3,
  TP_I32 = 4,
  TP_U32 = 5,
  TP_U8 = 6
} tp_dtype;

#define TP_MAX_RANK 8

/* Non-owning strided view of device (or host, where stated) memory. */
typedef struct tp_tensor {
  void* ptr;                      /* address of element (0, ..., 0)            */
  int32_t dtype;                  /* tp_dtype                                  */
  int32_t rank;                   /* 0 .. TP_MAX_RANK                          */
  int64_t shape[TP_MAX_RANK];     /* extents; only the first `rank` are read   */
  int64_t strides[TP_MAX_RANK];   /* element strides                           */
} tp_tensor;

typedef enum tp_map_kind {
  TP_MAP_IDENTITY = 0, /* plain partition: program p owns tile p (§3.4)         */
  TP_MAP_STRIDED = 1,  /* mapped: program p owns slots p, p+P, p+2P, ... (§3.6)  */
  TP_MAP_QUEUE = 2     /* mapped: a device counter hands out each slot once      */
} tp_map_kind;

typedef enum tp_mode {
  TP_SYNC = 0,    /* launch, synchronize the stream, release (§3.2 .sync())     */
  TP_ASYNC = 1,   /* launch, record `event`, return (§3.2 .await)               */
  TP_CAPTURE = 2  /* record into the graph open on `stream` (§3.2 .graph())     */
} tp_mode;

typedef struct tp_ctx tp_ctx;
typedef struct tp_partition tp_partition;
typedef struct tp_event tp_event;
typedef struct tp_graph tp_graph;

/* tp_exec.flags bits. */
enum {
  /* Device-checked launch (the debug build of a store, §3.6: a store is
   * validated against the partition map before it is made). Before storing
   * a tile, the storing program checks that the tile lies inside the
   * partition's grid and that the map gives it to this program, then claims
   * the tile in a bitmap held by the context; the launch's last claimant to
   * finish claiming clears the bitmap again, so the next launch and every
   * graph replay start from a clear bitmap with no extra node enqueued. A tile
   * that is off the grid, not the program's, or already claimed by another
   * program (two programs writing one sub-tensor: a data race, Appendix A)
   * is not stored, and the operation reports TP_ERR_RACE where it reports
   * device errors (SYNC: on return; ASYNC: from tp_event_query /
   * tp_event_wait; graph: from a SYNC replay or the replay's event).
   * Supported by the element-wise maps (tp_map_*), by tp_gemm and
   * tp_gemm_fp8 on the tensor-core path (tiles of 64, 128 or 256 rows) and by
   * tp_permute_heads_unchecked, up to 2^23 tiles per launch; other
   * operations return TP_ERR_UNSUPPORTED when it is set. The
   * bitmap and its finished-claimant counter are one per context: checked
   * launches of one context must not overlap in time (order them on one
   * stream), or they see each other's claims. */
  TP_EXEC_CHECKED = 1,
  /* Failure-path test hook of tp_gemm on 128-row tensor-core tiles: the
   * producer of every program leaves its first K block unloaded, so the MMA
   * issuer's bounded wait (cut to 50 ms) runs out; the kernel drains its
   * copies and MMAs, frees TMEM and returns, and the operation reports
   * TP_ERR_TIMEOUT where it reports device errors. C is left partly
   * written. Other operations, and 256-row tiles, return TP_ERR_UNSUPPORTED. */
  TP_EXEC_INJECT_TIMEOUT = 2,
  /* The decode products (tp_decode_norm_qkv_gu, tp_decode_down_residual):
   * the caller promises that no work queued before the call on its stream,
   * still running, writes the weight matrices (weights loaded once and
   * kept, as in a decode loop). The streaming kernel then starts copying
   * weights while the preceding kernels finish (this library's kernels let
   * the next one start early); its inputs h and a are still read only after
   * them. Without the flag every read waits for the preceding work. Other
   * operations return TP_ERR_UNSUPPORTED when it is set. */
  TP_EXEC_STATIC_WEIGHTS = 4
};

/* How an operation is executed. */
typedef struct tp_exec {
  int32_t mode;            /* tp_mode                                          */
  int32_t flags;           /* TP_EXEC_* bits; undefined bits must be 0         */
  void* stream;            /* cudaStream_t (borrowed); NULL = legacy stream    */
  tp_event* event;         /* ASYNC: event that completion is recorded into     */
  /* Optional write-count instrumentation (device pointers, NULL = off): each
   * store of output element i also adds 1 to write_counts[i] and writes the
   * storing program's id to write_owner[i]. Both arrays hold one entry per
   * output element in row-major order. Used by the partition checker
   * (Appendix A: each element written by exactly one program). */
  uint32_t* write_counts;
  int32_t* write_owner;
} tp_exec;

typedef struct tp_partition_info {
  int32_t rank;
  int32_t map_kind;        /* tp_map_kind                                      */
  int64_t shape[3];
  int64_t tile[3];
  int64_t grid[3];         /* ceil(shape / tile) per axis                      */
  int64_t num_tiles;
  int64_t num_programs;    /* = num_tiles for TP_MAP_IDENTITY                  */
  int32_t busy;            /* 1 while an operation on it is in flight          */
  int32_t reserved;
} tp_partition_info;

/* GEMM tile configuration (§5.1: tile shapes tuned per size). 0 = default. */
typedef struct tp_gemm_config {
  int32_t bm;          /* tensor-core GEMM: 64 or 128 (one CTA), or 256 (CTA
                        * pair, cta_group::2); SIMT GEMM: 64                   */
  int32_t bn;          /* 32..256, multiple of 32 (tensor-core paths)          */
  int32_t bk;          /* tensor-core GEMM: K per ring stage, 1, 2 or 4 K blocks
                        * of 128 bytes (64 bf16 / 128 fp8 elements; 0 = one).
                        * With more than one, each operand arrives as one 3-D
                        * TMA box per stage: fewer, larger copies (a copy
                        * costs about the same time whatever its size). The
                        * largest count up to bk that leaves room for two
                        * stages is used, and one block per stage when K is
                        * not a multiple of the K block or split_k > 1. The
                        * MMAs and their K order do not change, so C does
                        * not. SIMT GEMM: 8, 16 or 32.                       */
  int32_t stages;      /* shared-memory ring depth                              */
  int32_t group_m;     /* raster band height in tiles (L2 reuse)                */
  int32_t num_programs;/* persistent programs; 0 = number of SMs (or pairs)     */
  int32_t swap_ab;     /* compute C^T = B^T A^T. Grouped GEMM: per plan. BF16
                        * tensor-core tp_gemm: the partition's tiles are then
                        * W x 128 (W = 32, 64 or 128 rows of C); a CTA pair
                        * computes each as a 128 x W MMA tile whose rows are
                        * C's columns (64 rows of B^T per CTA) and whose
                        * columns are C's rows (W/2 rows of A per CTA), for
                        * short M, where a normal tile would leave most of
                        * the MMA's rows empty. No split_k, no narrow tiles
                        * in the last round; other values than 0 and 1 are
                        * reserved.                                           */
  int32_t split_k;     /* tensor-core GEMM, 128-row tiles: K slices per tile,
                        * 0 or 1 = none, 2, 4 or 8. A program is then a
                        * cluster of split_k CTAs; CTA s accumulates the K
                        * blocks [s*nk/split_k, (s+1)*nk/split_k) of the
                        * program's tile (nk = ceil(K / bk) >= split_k), and
                        * CTA j adds the split_k partial sums of column slice
                        * j (bn / split_k columns, a multiple of 32) in slice
                        * order and stores it, so every C element still has
                        * one writer and C is bit-reproducible (its rounding
                        * differs from split_k = 1). Needs at most one tile
                        * per program (an identity map, or a strided map with
                        * num_programs >= tiles). FP32 SIMT GEMM: 0, 1, 2
                        * or 4 CTAs per 64 x 64 tile program (not with a
                        * queue map); CTA r stores rows [r*64/S, +64/S) of
                        * the tile after adding the S partials in order.     */
  int32_t cut_limit;   /* tensor-core GEMM on a strided map with T tiles and P
                        * programs (split_k <= 1): each of the R = T mod P
                        * tiles of the last, partial round may be cut along N
                        * into S narrow tiles (S the largest power of two <=
                        * min(limit, P / R) leaving a multiple of 32 columns,
                        * 64 for 256-row tiles), run by programs that would
                        * otherwise idle in that round; every C element is
                        * still computed whole by one program, so C is
                        * bit-identical either way. Limit: 0 = 4 (default),
                        * 1 = never cut, 2..8. SIMT GEMM: ignored.           */
} tp_gemm_config;

/* ---------------------------------------------------------------- errors */
const char* tp_error_string(tp_status s);
/* Reason for the last non-OK status returned on this thread ("" if none). */
const char* tp_last_error_detail(void);
/* Library version (major, minor). 0.2: tp_gemm_config has the cut_limit
 * field (the last-round N-cut limit that split_k carried in 0.1) and
 * split_k selects split-K programs; tp_exec.flags has
 * TP_EXEC_INJECT_TIMEOUT. */
tp_status tp_version(int32_t* major, int32_t* minor);

/* --------------------------------------------------------------- context */
/* Creates a context on CUDA device `device` (§3.2 ExecutionContext: device,
 * stream and memory pool). Allocates the context's device workspace (error
 * word, queue counters, scale scratch) once, so later calls can be captured.
 * Errors: TP_ERR_INVALID (null out), TP_ERR_CUDA (no such device / no sm_103). */
tp_status tp_ctx_create(int32_t device, tp_ctx** out);
/* Frees the context and its workspace. TP_ERR_BUSY if work is still in flight. */
tp_status tp_ctx_destroy(tp_ctx* ctx);
/* Number of SMs and compute capability of the context's device. */
tp_status tp_ctx_info(tp_ctx* ctx, int32_t* sm_count, int32_t* cc_major, int32_t* cc_minor);

/* ---------------------------------------------------------------- tensors */
/* Fills a view (§3.3 Table 1 borrow rows; §3.2 TensorView). strides may be
 * NULL for a row-major contiguous layout. Errors: TP_ERR_INVALID (null view,
 * rank outside 0..8, negative extent, unknown dtype). */
tp_status tp_tensor_init(tp_tensor* t, void* ptr, int32_t dtype, int32_t rank,
                         const int64_t* shape, const int64_t* strides);
/* Zero-copy view of `base` (§3.2 TensorView: new shape, strides or slice over
 * the same allocation). `offset` is in elements from base->ptr. The view's
 * reachable elements must lie inside base's reachable range, else
 * TP_ERR_INVALID. */
tp_status tp_tensor_view(const tp_tensor* base, int64_t offset, int32_t rank,
                         const int64_t* shape, const int64_t* strides, tp_tensor* out);

/* ------------------------------------------------------------- partitions */
/* Partitions a contiguous mutable output into tiles of `tile` (one extent per
 * axis, §3.4): grid = ceil(shape / tile). Rank must be 1..3 (CUDA grids are
 * three-dimensional), else TP_ERR_RANK; tile extents must be >= 1, else
 * TP_ERR_INVALID. The partition starts as a plain partition (one program per
 * tile). The tensor's memory stays owned by the caller; the partition handle
 * is owned by the caller and freed with tp_partition_destroy. ctx may be NULL
 * to validate and inspect a partition on the host alone; such a partition
 * cannot be launched (operations return TP_ERR_INVALID). */
tp_status tp_partition_create(tp_ctx* ctx, const tp_tensor* out, const int64_t* tile,
                              tp_partition** p);
/* Turns p into a mapped partition (§3.6): `num_programs` programs walk the
 * tiles under map `kind`. TP_MAP_IDENTITY resets to a plain partition.
 * num_programs must be 1..num_tiles (§3.4: mapped partitions validate their
 * program count against the partition grid), else TP_ERR_INVALID.
 * TP_ERR_BUSY while in flight. */
tp_status tp_partition_map(tp_partition* p, int32_t kind, int64_t num_programs);
tp_status tp_partition_query(const tp_partition* p, tp_partition_info* info);
/* TP_ERR_BUSY while an operation on it is in flight. */
tp_status tp_partition_destroy(tp_partition* p);

/* ----------------------------------------------------------------- events */
/* Completion handle for TP_ASYNC operations (§3.2 .await; the host learns of
 * completion by polling or waiting instead of a driver callback). */
tp_status tp_event_create(tp_ctx* ctx, tp_event** ev);
/* *done = 1 once every operation recorded into ev has completed; then the
 * partitions those operations held are released and any device-side error
 * (TP_ERR_TIMEOUT) is reported. */
tp_status tp_event_query(tp_event* ev, int32_t* done);
/* Blocks until completion, releases the held partitions, reports errors. */
tp_status tp_event_wait(tp_event* ev);
/* TP_ERR_BUSY if it still holds partitions of unfinished work. */
tp_status tp_event_destroy(tp_event* ev);

/* ----------------------------------------------------------------- graphs */
/* Starts capturing `stream` into a new graph (§3.2 CudaGraph::scope). Ops
 * called with mode TP_CAPTURE on that stream are recorded, not run. One
 * capture per context at a time. */
tp_status tp_graph_begin(tp_ctx* ctx, void* stream, tp_graph** g);
/* Ends the capture and instantiates the graph. */
tp_status tp_graph_end(tp_graph* g);
/* Replays the graph with one launch (§5.2: one driver call for the whole
 * pipeline). The replay is itself an operation with a mode (SYNC or ASYNC,
 * §3.2): the partitions recorded into the graph are busy while it runs. */
tp_status tp_graph_replay(tp_graph* g, const tp_exec* ex);
/* *count = the kernel nodes of an ended graph (each replay launches that many
 * kernels). TP_ERR_INVALID before tp_graph_end; TP_ERR_CUDA if the graph
 * cannot be walked. */
tp_status tp_graph_kernel_count(tp_graph* g, int64_t* count);
tp_status tp_graph_destroy(tp_graph* g);

/* ----------------------------------------------------- element-wise maps */
/* z = alpha * x + y on every element (§2 Listing 1's element-wise add is
 * alpha = 1; §5.1 evaluates it at N = 2^28). z is a partition of an F32 or
 * BF16 contiguous tensor; x and y have z's shape and dtype. Arithmetic in fp32
 * (one fused multiply-add), BF16 output rounded to nearest even. Each tile
 * program stores only its own tile(s). Errors: TP_ERR_SHAPE, TP_ERR_ALIAS,
 * TP_ERR_BUSY, TP_ERR_UNSUPPORTED (non-contiguous), TP_ERR_CUDA. */
tp_status tp_map_axpy(tp_ctx* ctx, tp_partition* z, float alpha, const tp_tensor* x,
                      const tp_tensor* y, const tp_exec* ex);
/* y = gelu_tanh(x) * w, gelu_tanh(x) = 0.5 x (1 + tanh(sqrt(2/pi)(x + 0.044715 x^3)))
 * evaluated as x / (1 + exp(-2u)) with exp(-2u) = 2^(-2u log2 e) on the
 * hardware base-2 exponential; same layout rules as tp_map_axpy. */
tp_status tp_map_gelu_mul(tp_ctx* ctx, tp_partition* y, const tp_tensor* x,
                          const tp_tensor* w, const tp_exec* ex);
/* y = x * g element-wise (§5.2's pipeline kernel); same rules. */
tp_status tp_map_scale(tp_ctx* ctx, tp_partition* y, const tp_tensor* x, const tp_tensor* g,
                       const tp_exec* ex);
/* c <- c + a + b (§3.4 Listing 4: the mutable tile is read, then written by
 * the same program). */
tp_status tp_map_add_accum(tp_ctx* ctx, tp_partition* c, const tp_tensor* a,
                           const tp_tensor* b, const tp_exec* ex);

/* ------------------------------------------------------ head permutation */
/* Head permutation of a rank-4 attention tensor (§3.5, Listing 5), in units of
 * (BM, D) tiles: with src of shape (B, H, M, D) and M / BM == H,
 *   dst[b, m, h*BM + i, :] = src[b, h, m*BM + i, :]   (0 <= m, h < H, 0 <= i < BM),
 * i.e. destination tile (b, m, h) is source tile (b, h, m).
 * tp_permute_heads is the partitioned form (§3.5): `dst` is a plain partition
 * of the F32 output viewed as (B*H, M, D) with tiles (1, BM, D); program t
 * stores only sub-tensor t, so no destination index is chosen in the kernel.
 * `src` is a contiguous F32 tensor (B, H, M, D), not overlapping dst.
 * Errors: TP_ERR_SHAPE (M % BM, M / BM != H, tiles not (1, BM, D)),
 * TP_ERR_ALIAS, TP_ERR_BUSY, TP_ERR_UNSUPPORTED (non-contiguous, mapped
 * partition), TP_ERR_CUDA. */
tp_status tp_permute_heads(tp_ctx* ctx, tp_partition* dst, const tp_tensor* src, int64_t H, const tp_exec* ex);
/* The same permutation written against raw device pointers (the unchecked
 * escape hatch of §3.6), launched with Listing 5's grid (B*H, H, 1):
 * program (bh1, h2), b = bh1 / H, h1 = bh1 % H, loops m over the H source
 * tiles and stores source tile (b, h1, m) at destination tile (b, m, hd) with
 * hd = h2 when `swap_bug` is non-zero (Listing 5's swapped index) and hd = h1
 * otherwise (then only the programs with h2 == 0 store). With swap_bug, the H
 * programs that differ in h1 store to the same destination tile: a data race
 * whose surviving values are unordered; the write counts report H writes per
 * element (program id = bh1 * H + h2). dst and src: contiguous F32
 * (B, H, M, D) device buffers that must not overlap; M / BM == H keeps every
 * store in bounds. `ex` gives the stream, the mode (no partition is held, so
 * nothing becomes busy), the optional write counts and TP_EXEC_CHECKED: the
 * checked launch lets only the first program that claims a destination tile
 * store it and reports TP_ERR_RACE when any claim was refused.
 * Errors: TP_ERR_SHAPE, TP_ERR_INVALID, TP_ERR_ALIAS, TP_ERR_RACE, TP_ERR_CUDA. */
tp_status tp_permute_heads_unchecked(tp_ctx* ctx, void* dst, const void* src, int64_t B, int64_t H, int64_t M,
                                     int64_t D, int64_t BM, int32_t swap_bug, const tp_exec* ex);

/* ------------------------------------------------------------------ GEMM */
/* C = A . B with one C tile per program and a K loop (§3.6 Listing 6).
 * c: partition of a row-major M x N output whose tile is the GEMM tile.
 * a: M x K. b: K x N (its strides decide the layout: row stride 1 means B is
 * stored N x K, "K-major").
 * - F32 A, B, C: FFMA tiles of 64 x 64 (no TF32), any strides. With bk = 32
 *   (the default), row-major A and B whose row pitches are multiples of 4
 *   floats and whose bases are 16-byte aligned, and an identity or strided
 *   map (split programs holding one tile each), the operands are brought by
 *   TMA; otherwise each thread stages them through registers. Both give
 *   the same C bit for bit.
 * - BF16 A, B, C: tcgen05 tensor-core path. A must be K-major (row-major
 *   M x K) and B K-major (stored N x K); base addresses 16-byte aligned and
 *   K a multiple of 8 (TMA rows are 16-byte multiples), else TP_ERR_ALIGN.
 *   FP32 accumulation in tensor memory; C rounded to bf16 (nearest even).
 *   Tiles of 64 or 128 rows run on one CTA (64: tcgen05 M = 64, for short
 *   M), 256 rows on a CTA pair; columns 32..256, a multiple of 32 (64 for
 *   256 rows). c's tile must be (cfg.bm, cfg.bn) or (128, bn) for the
 *   default config.
 * cfg may be NULL (defaults). The partition may be plain or mapped
 * (TP_MAP_STRIDED: persistent programs). Errors: TP_ERR_SHAPE, TP_ERR_ALIGN,
 * TP_ERR_ALIAS, TP_ERR_BUSY, TP_ERR_UNSUPPORTED, TP_ERR_TIMEOUT, TP_ERR_CUDA. */
tp_status tp_gemm(tp_ctx* ctx, tp_partition* c, const tp_tensor* a, const tp_tensor* b,
                  const tp_gemm_config* cfg, const tp_exec* ex);

/* How many programs of the tensor-core GEMM can be resident on the device at
 * once for `cfg` (bm 64, 128 or 256, bn, stages; 0 fields take the
 * defaults): CTA pairs for 256-row tiles, CTAs otherwise. A
 * persistent launch with more programs than this runs the extra ones after
 * others finish. With split_k > 1 the count is of split programs (clusters
 * of split_k CTAs); with swap_ab of CTA pairs. Errors: TP_ERR_INVALID,
 * TP_ERR_UNSUPPORTED, TP_ERR_CUDA. */
tp_status tp_gemm_resident_programs(tp_ctx* ctx, const tp_gemm_config* cfg, int32_t* programs);

/* The BF16 tensor-core GEMM against a raw output pointer: the unchecked
 * baseline of §5.1 (the same schedule with manual raw-pointer output access).
 * `c` is a contiguous BF16 M x N device buffer; A and B as for tp_gemm.
 * cfg->bm (64, 128 or 256) and cfg->bn give the tile (with cfg->swap_ab: W =
 * 32, 64 or 128 rows x 128 columns, on CTA pairs); cfg->num_programs > 0
 * maps tiles strided over that many programs (CTA pairs for bm = 256), 0
 * launches one program per tile; cfg->stages and cfg->group_m as for tp_gemm.
 * No partition is involved: nothing is checked against aliasing or work in
 * flight and nothing is marked busy; the call only enqueues on `stream`.
 * Errors: TP_ERR_INVALID, TP_ERR_RANK, TP_ERR_SHAPE, TP_ERR_ALIGN,
 * TP_ERR_UNSUPPORTED, TP_ERR_CUDA. */
tp_status tp_gemm_unchecked(tp_ctx* ctx, void* c, const tp_tensor* a, const tp_tensor* b, const tp_gemm_config* cfg,
                            void* stream);

/* ------------------------------------------------ FP8-E4M3 GEMM pipeline */
/* Per-tensor-scaled FP8 GEMM (the FP8 workload; the paper's GEMM of §3.6 /
 * §5.1 is f16): amax -> scale -> quantise -> tcgen05 kind::f8f6f4 GEMM with
 * FP32 accumulation and an FP32 dequantising epilogue.
 *
 * tp_amax: *amax (device float) = max |x| over every element of the
 * contiguous F32/BF16 tensor x (0 for an empty or all-zero tensor). The
 * reduction uses atomic max on a single word, so it is not a partitioned
 * output; *amax is cleared on the stream first. */
tp_status tp_amax(tp_ctx* ctx, const tp_tensor* x, float* amax, const tp_exec* ex);
/* q = E4M3(satfinite(RN(x * s))) with s = 448 / *amax in fp32 (s = 1 when
 * *amax = 0); *scale (device float) receives s. q is a partition of an
 * F8E4M3 (or U8) tensor with x's shape whose tiles span whole rows (rank 2:
 * tile = [rows, K]); x is contiguous F32 or BF16. Codes are bit-exact
 * functions of x and *amax (the product is an fp32 multiply). */
tp_status tp_quantize_fp8(tp_ctx* ctx, tp_partition* q, const tp_tensor* x, const float* amax, float* scale,
                          const tp_exec* ex);
/* C (bf16) = (qA . qB) * 1 / (*scale_a * *scale_b) (dequantisation factor in
 * fp32). qA: M x K E4M3, K-major; qB: K x N E4M3 view of N x K storage
 * (K-major); K a multiple of 16. Same tiles, maps, configs and errors as the
 * BF16 path of tp_gemm (128 K elements per pipeline stage). */
tp_status tp_gemm_fp8(tp_ctx* ctx, tp_partition* c, const tp_tensor* qa, const tp_tensor* qb,
                      const float* scale_a, const float* scale_b, const tp_gemm_config* cfg, const tp_exec* ex);

/* ------------------------------------------------------ grouped GEMM */
/* One problem of a group: C = A . B (BF16 in and out, FP32 accumulation).
 * a: M x K, K-major (row-major); b: K x N view of N x K storage (K-major);
 * c: contiguous M x N. Device pointers; K a multiple of 8; 16-byte aligned. */
typedef struct tp_gemm_problem {
  tp_tensor a;
  tp_tensor b;
  tp_tensor c;
} tp_gemm_problem;

typedef struct tp_grouped_plan tp_grouped_plan;

/* Plans a group of 1..65536 independent GEMMs for one persistent launch (the
 * many-uneven-GEMMs workload; the paper's nearest setting is its bimodal GEMM
 * queue, Appendix B). Every output tile of every problem becomes one slot of
 * a device queue, most expensive tiles first. Problems with M <= swap_max_m
 * (<= 256; a negative value means 256) run transposed, C^T = B^T . A^T, with
 * tiles spanning all of M; the others use tiles of 256 columns. cta_pair != 0
 * runs every tile on a CTA pair (tcgen05 cta_group::2, 256 tile rows in the
 * MMA orientation), 0 on single CTAs (128 rows). The plan owns one
 * queue-mapped partition per C_i and a device table of TMA descriptors; it
 * allocates device memory, so build it outside graph capture
 * (TP_ERR_CAPTURE). Errors: TP_ERR_RANK, TP_ERR_SHAPE, TP_ERR_ALIGN,
 * TP_ERR_UNSUPPORTED, TP_ERR_CUDA. */
tp_status tp_grouped_plan_create(tp_ctx* ctx, const tp_gemm_problem* probs, int32_t n, int32_t swap_max_m,
                                 int32_t cta_pair, tp_grouped_plan** plan);
/* Total queue slots, and per problem (input order) whether it runs
 * transposed (swapped may be NULL). */
tp_status tp_grouped_plan_info(const tp_grouped_plan* plan, int64_t* total_tiles, int32_t* swapped);
/* TP_ERR_BUSY while a launch of the plan is in flight. */
tp_status tp_grouped_plan_destroy(tp_grouped_plan* plan);
/* Runs the whole group with one launch of num_programs persistent programs
 * (CTAs, or CTA pairs; 0 = one per SM / SM pair) that dequeue tiles until
 * the queue is empty. Every C_i is
 * busy while in flight. Write-count instrumentation indexes the C_i back to
 * back in input order (C_0's elements first). Errors: as tp_gemm. */
tp_status tp_grouped_gemm(tp_ctx* ctx, tp_grouped_plan* plan, int32_t num_programs, const tp_exec* ex);

/* --------------------------------------------------- decode-shaped chain */
/* One layer of a batch-1 decode forward pass (§3.2, Listing 3: RMSNorm,
 * matrix-vector products and a residual add, captured once and replayed),
 * widened to a gated MLP. Vectors are contiguous FP32 rank-1 tensors;
 * weights are BF16 [out, in] row-major with rows 16-byte aligned. Every
 * output vector is a partition (rank 1); each row is written by one program.
 *
 * n = h / sqrt(mean(h^2) + eps) * gamma (gamma may be NULL: 1). */
tp_status tp_rmsnorm(tp_ctx* ctx, tp_partition* n_out, const tp_tensor* h, const tp_tensor* gamma, float eps,
                     const tp_exec* ex);
/* y = W x (W [rows, k] bf16, x [k] fp32, y [rows] fp32, FP32 accumulation). */
tp_status tp_gemv(tp_ctx* ctx, tp_partition* y, const tp_tensor* w, const tp_tensor* x, const tp_exec* ex);
/* a = silu(g) * u for gu = [g; u] (gu has 2n entries, a has n). */
tp_status tp_silu_mul(tp_ctx* ctx, tp_partition* a_out, const tp_tensor* gu, const tp_exec* ex);
/* h <- h + d (the residual add; h is read and written by its own program). */
tp_status tp_residual_add(tp_ctx* ctx, tp_partition* h, const tp_tensor* d, const tp_exec* ex);
/* Fused: n = rmsnorm(h) (recomputed by every program), qkv = W_qkv n and
 * a = silu(W_gu[:ni] n) * (W_gu[ni:] n), in one launch. Write counts index
 * qkv's rows, then a's. */
tp_status tp_decode_norm_qkv_gu(tp_ctx* ctx, tp_partition* qkv, tp_partition* a_out, const tp_tensor* h,
                                const tp_tensor* gamma, const tp_tensor* w_qkv, const tp_tensor* w_gu, float eps,
                                const tp_exec* ex);
/* Fused: h <- h + W_down a, in one launch. */
tp_status tp_decode_down_residual(tp_ctx* ctx, tp_partition* h, const tp_tensor* w_down, const tp_tensor* a_in,
                                  const tp_exec* ex);

/* ------------------------------------------------------------ autotuner */
/* Tile-configuration search for the tensor-core GEMM (§5.1 tunes tile shapes
 * once per size; the algorithm and its numerics stay fixed).
 *
 * Numerics classes. Every config with split_k <= 1 computes each C element
 * as one FP32 accumulation over K, in K order, by the one program that owns
 * its tile; tile rows, tile columns, K per stage, stages, raster band and
 * program count only decide where and when that happens. All such configs, and the default
 * config (cfg NULL), therefore give bit-identical C: the single-pass class.
 * A split-K config adds split_k slice partials in slice order instead:
 * reproducible, but rounded differently. Searches cover the single-pass
 * class unless the caller opts in to split-K with TP_TUNE_SPLIT_K, so a
 * tuned or proposed config never changes C unless asked to. */
enum {
  TP_TUNE_SPLIT_K = 1, /* also search the split-K configs (changes C's rounding) */
  TP_TUNE_SWAP_AB = 2  /* also search the swap-AB configs (single-pass class;
                        * tried on BF16 problems of at most W rows). Measured
                        * on skinny shapes they ran within a few per cent of
                        * 64-row tiles, and adding them to the proposer's
                        * outputs raised its p90 regret, so the default
                        * search and the proposer leave them out. */
};
/* The space (same order on every call; with flags = 0, index i is the MLP
 * proposer's output i): tile rows {64, 128 (one CTA), 256 (CTA pair)} x tile
 * columns {64, 128, 192, 256} x K per stage {1, 2, 4} K blocks (bk; the
 * deepest ring that fits) x raster bands {1, 8}, the 72 single-pass configs;
 * with TP_TUNE_SPLIT_K followed by the split-K programs of 128-row tiles:
 * (bn 128, split_k 2 / 4) and (bn 256, split_k 2 / 4 / 8). TP_TUNE_SWAP_AB
 * inserts, after the 72, the swap-AB configs: W x 128 C tiles (bm = W = 32,
 * 64, 128; bn 128; swap_ab 1) x K per stage {2, 4} K blocks. Writes up to `cap` configs to `out` (may be NULL) and the size
 * to *count. Errors: TP_ERR_INVALID (undefined flag bits), TP_ERR_UNSUPPORTED
 * (dtype). */
tp_status tp_autotune_space(int32_t dtype, int32_t flags, tp_gemm_config* out, int32_t cap, int32_t* count);
/* Times every config of tp_autotune_space(dtype, flags) on an M x N x K
 * problem of `dtype` (TP_BF16 or TP_F8E4M3; K * element size a multiple of
 * 16) held in a device workspace the context owns (grown with cudaMalloc:
 * not during capture, TP_ERR_CAPTURE), `reps` back-to-back launches per
 * config timed with CUDA events (0 = 2..10 by problem size). Split-K configs
 * are skipped (0 TFLOP/s) when the shape's tiles x split_k exceed twice the
 * SM count or K has fewer than split_k blocks. Returns the fastest config
 * (ties within 1% keep the earlier one), optionally the TFLOP/s of every
 * config (space order) and the best TFLOP/s, and caches the winner under
 * (M, N, K, dtype, flags). */
tp_status tp_autotune(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, int32_t reps, int32_t flags,
                      tp_gemm_config* best, float* tflops_per_config, float* best_tflops);
/* Re-times one config on the autotuner's workspace problem of that shape:
 * `repeats` (1..64) independent timings of `reps` back-to-back launches
 * (0 = as tp_autotune), each after a delay kernel that lets the host queue
 * them all; *tflops_median = the median TFLOP/s. A split-K cfg is timed as
 * given. Errors as tp_autotune, plus the launch's own (a config that cannot
 * run on the shape). */
tp_status tp_autotune_time(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, const tp_gemm_config* cfg,
                           int32_t reps, int32_t repeats, float* tflops_median);
/* Cached winner of a search with `flags` for (M, N, K, dtype): *found = 1
 * and *out filled, else 0. */
tp_status tp_autotune_lookup(tp_ctx* ctx, int64_t M, int64_t N, int64_t K, int32_t dtype, int32_t flags,
                             tp_gemm_config* out, int32_t* found);
/* Persist / restore the cache (text, "tp-autotune-cache v5": one line per
 * entry, M N K dtype flags bm bn bk stages group_m num_programs split_k
 * swap_ab TFLOP/s). Load also reads v4 files (no swap_ab column: 0), v3
 * files (no bk column: bk 0) and v2 and v1
 * files (no flags column; v1 lines also lack split_k), whose searches
 * covered the split-K configs: an entry is filed under TP_TUNE_SPLIT_K, and
 * a single-pass winner under flags 0 too. */
tp_status tp_autotune_save(tp_ctx* ctx, const char* path);
tp_status tp_autotune_load(tp_ctx* ctx, const char* path);

/* ------------------------------------------------- learned tile proposer */
/* A 3-layer ReLU MLP (in -> hidden -> hidden -> out) trained on the GPU by
 * the library's own kernels. Parameters are one fp32 buffer
 * [W1 (hidden x in), b1, W2 (hidden x hidden), b2, W3 (out x hidden), b3],
 * matrices row-major [out, in]. Loss: sum V (y - T)^2 / max(1, sum V) over a
 * batch (V masks invalid entries); optimiser: Adam (0.9, 0.999, 1e-8) with
 * bias correction. X, T, V, Y, loss and grads are device pointers; X is
 * [batch, in], T, V, Y are [batch, out]. The tp_mlp object owns its
 * parameters, optimiser state and scratch; calls on one tp_mlp must be
 * ordered on one stream (tp_exec.stream; SYNC waits, ASYNC returns). */
typedef struct tp_mlp tp_mlp;
/* Creates an MLP with in, hidden, out <= 1024 units (in >= 1) for batches of
 * up to max_batch rows, parameters copied from the host array init_params
 * (layout above); allocates device memory, so not during graph capture
 * (TP_ERR_CAPTURE). Errors: TP_ERR_INVALID, TP_ERR_CAPTURE, TP_ERR_CUDA. */
tp_status tp_mlp_create(tp_ctx* ctx, int32_t in, int32_t hidden, int32_t out, int32_t max_batch,
                        const float* init_params, tp_mlp** mlp);
/* Frees the MLP and its device memory (no work of it may be in flight). */
tp_status tp_mlp_destroy(tp_mlp* mlp);
/* Number of fp32 parameters (the length of the parameter layout above). */
tp_status tp_mlp_num_params(const tp_mlp* mlp, int64_t* count);
/* Copies the parameters to the host array host_out (synchronous). */
tp_status tp_mlp_get_params(const tp_mlp* mlp, float* host_out);
/* Sets the parameters (host array) and resets the optimiser state. */
tp_status tp_mlp_set_params(tp_mlp* mlp, const float* host_in);
tp_status tp_mlp_forward(tp_mlp* mlp, const float* X, int32_t batch, float* Y, const tp_exec* ex);
/* Forward, loss (*loss, may be NULL) and gradient of every parameter
 * (copied to grads when not NULL). */
tp_status tp_mlp_loss_grad(tp_mlp* mlp, const float* X, const float* T, const float* V, int32_t batch,
                           float* loss, float* grads, const tp_exec* ex);
/* tp_mlp_loss_grad followed by one Adam step at learning rate lr. */
tp_status tp_mlp_train_step(tp_mlp* mlp, const float* X, const float* T, const float* V, int32_t batch,
                            float lr, float* loss, const tp_exec* ex);
/* Persist / restore the parameters and sizes as text ("tp-mlp v1"); load
 * requires matching sizes (TP_ERR_SHAPE) and resets the optimiser state.
 * Errors: TP_ERR_INVALID (unreadable / malformed file), TP_ERR_SHAPE. */
tp_status tp_mlp_save(const tp_mlp* mlp, const char* path);
tp_status tp_mlp_load(tp_mlp* mlp, const char* path);
/* Proposer features of a shape: [log2 M, log2 N, log2 K, BF16?, FP8?] (host). */
tp_status tp_mlp_features(int64_t M, int64_t N, int64_t K, int32_t dtype, float* out);
/* Training targets of one autotuner table: target_i = max(tflops_i, 0) /
 * max tflops and mask_i = 1 (a config that did not run scores 0), or all
 * masked (0) when no config ran (host arrays of `count`). */
tp_status tp_mlp_targets(const float* tflops, int32_t count, float* target, float* mask);
/* Proposes a config for (M, N, K, dtype): the MLP's arg-max over the
 * single-pass configs (tp_autotune_space with flags 0; ties: lowest index).
 * Falls back to the exhaustive autotuner over the same class (cached; flags
 * 0) when the best score is below min_score or a dimension exceeds 16384
 * (outside the trained range); *used_fallback tells which. Proposal and
 * fallback choose within one numerics class, so C is bit-identical to the
 * default config's whichever they pick: a proposal never changes numerics. */
tp_status tp_propose(tp_ctx* ctx, tp_mlp* mlp, int64_t M, int64_t N, int64_t K, int32_t dtype, float min_score,
                     tp_gemm_config* out, float* score, int32_t* used_fallback);

/* ------------------------------------------------------------ diagnostics */
/* Exercises the failure path every pipelined kernel (the tensor-core GEMMs,
 * the grouped GEMM) relies on: one GPU thread waits on a shared-memory
 * mbarrier with the same bounded wait those kernels' roles use. With
 * arrive != 0 the barrier is signalled first and the wait completes (TP_OK).
 * With arrive == 0 nothing ever signals it: the wait gives up after
 * `limit_ns` of GPU wall time (1e3..2e9), records a timeout in the context's
 * error word and the kernel returns, so the operation reports TP_ERR_TIMEOUT
 * where it reports device errors (SYNC: on return; ASYNC: from
 * tp_event_query / tp_event_wait; graph: from the replay) and the context
 * stays usable. No output is involved, so nothing becomes busy. */
tp_status tp_diag_bounded_wait(tp_ctx* ctx, int64_t limit_ns, int32_t arrive, const tp_exec* ex);

/* ------------------------------------------------- allocation-free entry */
/* Queue-mapped z = alpha * x + y that needs no context and allocates nothing.
 * The paper has no counterpart. It exists for callers that cannot call
 * cudaMalloc: code inside a runtime or plugin whose device memory is wholly
 * owned by the host application's arena allocator (an allocation of its own
 * would bypass that budget, and fails once the arena holds the device), and
 * code on a latency-critical path where cudaMalloc / cudaFree are not
 * allowed because they can synchronise the device. Such a caller passes only
 * its inputs and output:
 *   z, x, y       device pointers to n contiguous elements of `dtype`
 *                 (TP_F32 or TP_BF16); x and y must not overlap z.
 *   tile          elements per tile (>= 1); the output is split into
 *                 ceil(n / tile) tiles that a device queue hands out, each
 *                 exactly once, to `num_programs` persistent programs
 *                 (1..number of tiles).
 *   stream        cudaStream_t (NULL = legacy stream); the call only enqueues.
 * The result equals tp_map_axpy on a TP_MAP_QUEUE partition, bit for bit.
 * Scratch: the queue's one 32-bit tile counter, kept in a static device array
 * of 256 bytes that every GPU loading this library holds until exit. The
 * first call on a device does that device's set-up with the device current:
 * it looks up the array's device address and loads the kernels this entry
 * point launches. Make that first call on each device before any stream
 * capture. Each call clears the counter on `stream` before its launch, in
 * stream order behind earlier work on that stream. All calls share the
 * counter: calls that overlap on the GPU (on different streams without
 * ordering between them) race on it and may skip or repeat tiles, so order
 * such calls with one stream or with events.
 * Limit: at most 2^31 tiles (TP_ERR_INVALID beyond). Errors: TP_ERR_INVALID
 * (bad sizes, null pointers), TP_ERR_ALIAS, TP_ERR_UNSUPPORTED (dtype),
 * TP_ERR_CUDA. Calls cudaMalloc, cudaFree or any allocating routine never. */
tp_status tp_map_axpy_queue_noalloc(void* z, const void* x, const void* y, int32_t dtype, int64_t n,
                                    int64_t tile, int32_t num_programs, float alpha, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* TP_H */
