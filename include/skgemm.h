/*
 * skgemm -- Stream-K GEMM for NVIDIA GB300 (sm_103a), C ABI.
 *
 * Operation (paper, Introduction and Background: general matrix-matrix
 * multiplication decomposed across GPU cores):
 *
 *     C = alpha * A * B + beta * C_in          A: m x k, B: k x n, C: m x n
 *
 * The MAC-loop iterations of all output tiles are split across persistent
 * units -- one CTA, or a pair of CTAs sharing a 256-row tile, per SM or
 * per SM pair ("Stream-K", the work-centric decomposition the paper
 * studies; Introduction, Background, Methodology, after Osama et al.,
 * PPoPP 2023).  Tiles that are cut between units spill FP32 partials to a
 * caller-provided workspace; the unit that holds the tile's first k-block
 * (its owner) waits on per-CTA flags and adds the partials in ascending unit
 * order (or, with SK_FIXUP_LAST_ARRIVER, the last unit to arrive adds them
 * in that same order), so the result is bit-reproducible for a fixed
 * problem, config and unit count.  A hybrid mode computes whole tiles in data-parallel waves
 * (Background, Fig. 1) and only the ragged remainder Stream-K.  Ragged
 * M, N and K are handled without padding (Results: the padding study).
 *
 * Conventions for every entry point:
 *  - All pointers to matrices, scales and workspace are DEVICE pointers of
 *    the current device; problem/config structs are HOST memory, read only
 *    during the call.  The library never allocates device memory and keeps
 *    no pointer after returning.
 *  - Launches are asynchronous on `stream` (NULL = legacy default stream);
 *    nothing synchronises the host except sk_get_status.
 *  - Host-detectable errors return before anything is launched.  A device
 *    side error (a bounded fixup wait that expired) is recorded in the
 *    workspace's status word and read back with sk_get_status; the output
 *    is then undefined.
 *  - The first call on a device resolves device attributes and the driver's
 *    tensor-map encoder; make it before capturing a stream into a CUDA graph.
 */
#ifndef SKGEMM_H
#define SKGEMM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SK_API __attribute__((visibility("default")))
#else
#define SK_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so no CUDA header is needed. */
typedef struct CUstream_st *sk_stream_t;

typedef enum {
    SK_OK = 0,
    SK_ERR_INVALID_ARG = 1,         /* null pointer, negative size, bad enum, ld too small */
    SK_ERR_UNSUPPORTED = 2,         /* valid but not implemented (dtype combo, alignment) */
    SK_ERR_WORKSPACE_TOO_SMALL = 3, /* ws_bytes < sk_workspace_size() */
    SK_ERR_TIMEOUT = 4,             /* a bounded device wait expired (from sk_get_status) */
    SK_ERR_CUDA = 5,                /* a CUDA runtime/driver call failed */
    SK_ERR_NO_DEVICE = 6            /* no CUDA device / architecture not sm_103 */
} sk_status;

typedef enum { SK_F32 = 0, SK_BF16 = 1, SK_E4M3 = 2 } sk_dtype;
typedef enum { SK_ROW_MAJOR = 0, SK_COL_MAJOR = 1 } sk_layout;

/* Work decomposition (paper, Background and Future Work; Osama et al.).
 *  DP      : one whole output tile per CTA per wave.
 *  SK      : all MAC-loop iterations of all tiles split evenly over the CTAs.
 *  HYBRID1 : (tiles mod CTAs) tiles Stream-K, the rest in whole DP waves.
 *  HYBRID2 : (CTAs + tiles mod CTAs) tiles Stream-K ("two-tile" Stream-K),
 *            the rest in whole DP waves; all Stream-K when tiles <= CTAs.
 *  AUTO    : the library's choice: the mode (and, if left 0, the tile) its
 *            runtime model predicts fastest for the problem set.          */
typedef enum {
    SK_MODE_AUTO = 0,
    SK_MODE_DP = 1,
    SK_MODE_SK = 2,
    SK_MODE_HYBRID1 = 3,
    SK_MODE_HYBRID2 = 4
} sk_mode;

/* One GEMM.  Element (i, j) of a row-major matrix X with leading dimension
 * ldx lives at X[i * ldx + j]; of a column-major one at X[i + j * ldx].
 * ld must be >= the contiguous extent.
 * Supported type combinations:
 *   A,B F32  -> C F32               (SIMT FFMA kernel, any layouts)
 *   A,B BF16 -> C BF16 or F32       (tcgen05 kernel; FP32 accumulate)
 *   A,B E4M3 -> C BF16 or F32       (tcgen05 kernel; FP32 accumulate;
 *                                    A row-major and B column-major only)
 * For BF16/E4M3 the TMA engine needs every base address 16-byte aligned and
 * lda/ldb times the element size a multiple of 16 bytes (else UNSUPPORTED).
 * C_in may equal C; it is read only when beta != 0 and must then have C's
 * type, layout and ldc.  scale_a / scale_b (E4M3 only; NULL means 1.0) are
 * device pointers to one float each, multiplied into alpha on the device. */
typedef struct {
    int64_t m, n, k;
    sk_dtype a_type, b_type, c_type;
    sk_layout a_layout, b_layout, c_layout;
    int64_t lda, ldb, ldc;
    const void *A;
    const void *B;
    const void *C_in;
    void *C;
    float alpha, beta;
    const float *scale_a;
    const float *scale_b;
} sk_problem;

/* How a tile split across units gets its partial sums added (Stream-K's
 * "fixup", Background and Methodology sections).  Every protocol adds in the
 * same order -- the partial of the unit holding k-block 0 first, then the
 * other units' partials by ascending unit index -- so all give bit-identical
 * C (with two partials the single addition is order-free). */
typedef enum {
    SK_FIXUP_OWNER = 0,        /* the unit holding k-block 0 waits (bounded) for
                                  the others' flags and adds their partials */
    SK_FIXUP_LAST_ARRIVER = 1, /* every contributor spills its partial and counts
                                  its arrival with one atomic; the contributor that
                                  completes the count adds all partials.  No unit
                                  ever waits; the workspace holds twice the partial
                                  slots (no counterpart in the paper) */
    SK_FIXUP_SPLIT = 2,        /* for plans where every unit holds one range inside
                                  one tile (all Stream-K, equal ranges dividing the
                                  tiles' k-blocks; otherwise SK_ERR_UNSUPPORTED):
                                  every contributor spills and waits (bounded) for
                                  the others, then sums its share of the tile from
                                  all partials in the same order and stores it.
                                  With the fixup left at SK_FIXUP_OWNER and the unit
                                  count left to the library, the library uses it
                                  where its runtime model predicts a gain (no
                                  counterpart in the paper) */
    SK_FIXUP_SPLIT_CLUSTER = 3 /* the split reduce for plans that cut every tile
                                  into k = 2, 4 or 8 equal tile-aligned ranges (k
                                  units per tile, at most 8 CTAs): the tile's k
                                  units run as one thread-block cluster and each
                                  writes the parts of its partial that the others
                                  sum straight into their shared memories -- no
                                  workspace slots or flags.  Single-problem BF16
                                  or 3xTF32 calls on 128-row tiles or 256 x 256
                                  pairs; otherwise SK_ERR_UNSUPPORTED.  The
                                  library picks it by itself (like SK_FIXUP_SPLIT)
                                  with k = 2 and one co-resident cluster per tile
                                  (no counterpart in the paper) */
} sk_fixup;

/* Kernel for FP32 problems. */
typedef enum {
    SK_F32_AUTO = 0,       /* 3xTF32 where every problem allows it (A row-major,
                              B column-major after normalising C to row-major,
                              16-byte aligned bases and leading dimensions),
                              otherwise FFMA */
    SK_F32_FFMA = 1,       /* FP32 fused multiply-add on the SIMT pipes:
                              128 x 128 tiles, 16-deep k-blocks */
    SK_F32_TF32X3 = 2      /* tensor cores: each operand x = x_hi + x_lo with
                              x_hi = x truncated to TF32 (as the MMA reads an
                              FP32 container), x_lo = tf32(x - x_hi), and
                              a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi accumulated
                              in FP32 (dropped a_lo b_lo and the rounding of the
                              low parts: at most about 2^-19 |a b| per product,
                              measured 3.3e-7 of sum |a||b|); 128 x
                              128 tiles, 32-deep k-blocks, K-major operands
                              only, else SK_ERR_UNSUPPORTED */
} sk_f32_kernel;

/* Launch configuration.  Zero in any field selects the default. */
typedef struct {
    int tile_m;              /* 128, or 256 = CTA-pair kernel (two CTAs of a cluster
                                share one 256 x tile_n tile through tcgen05
                                cta_group::2; BF16 and E4M3); 0 = chosen by the
                                library's runtime model */
    int tile_n;              /* F32: 128; BF16/E4M3: 128 or 256; pair: 256, 128 (BF16)
                                or 512 (BF16/E4M3, one problem: two N = 256 MMAs per
                                k-step into one 512-column TMEM accumulator, no
                                epilogue overlap); 0 = chosen by the library's
                                runtime model (512 only for data-parallel plans) */
    int stages;              /* smem pipeline depth (BF16/E4M3: 2..6; default by tile) */
    sk_mode mode;            /* decomposition; default AUTO */
    int num_ctas;            /* persistent CTAs, 1 <= num_ctas <= SM count; 0 = SM count,
                                or, when the library chooses the tile or the mode
                                and the problem has fewer tiles than units, possibly
                                a multiple of the tile count (every tile then splits
                                into equal parts).  The pair kernel uses num_ctas / 2
                                pairs, at most as many as the GPU can hold at once */
    int min_iters_per_unit;  /* fewest k-blocks per Stream-K unit; default 4 */
    uint64_t timeout_ns;     /* bound on every device-side wait; default 2e9 ns */
    int debug_flags;         /* test-only fault injection, 0 in normal use:
                                bit 0 = peers never raise their flags (owner
                                protocol) or count their arrival (split reduce),
                                so the others' bounded waits expire
                                (SK_ERR_TIMEOUT); the last-arriver protocol has no
                                wait.  With bit 0 set the library never picks the
                                split reduce by itself. */
    uint64_t *trace;         /* optional DEVICE buffer of SK_TRACE_BYTES_PER_CTA
                                bytes per launched CTA (single-problem BF16 and
                                3xTF32 calls; ignored elsewhere):
                                each CTA records its timeline there, see
                                SK_TRACE_* below; NULL = no tracing */
    int raster_group;        /* tile rows walked together by the rasterisation
                                (L2 locality of concurrently running tiles);
                                0 = default 8, at most 64 */
    sk_fixup fixup;          /* partial-sum fixup protocol; default SK_FIXUP_OWNER */
    sk_f32_kernel f32_kernel;/* FP32 problems only; default SK_F32_AUTO */
    uint32_t *coverage;      /* optional DEVICE buffer of sk_plan_info.coverage_words
                                words, zeroed by the caller: the kernel counts
                                which unit ran each MAC-loop iteration and which
                                unit stored each 32 x 32 block of C (layout
                                under SK_COVERAGE below).  Tensor-core kernels
                                only (BF16 single and grouped, FP32 as 3xTF32
                                single); ignored elsewhere.  A debug variant:
                                NULL = the normal kernels run */
} sk_config;

/* Coverage counts (sk_config.coverage), after the schedule the paper's
 * Background and Methodology describe: every (tile, k-block) MAC-loop
 * iteration is computed by exactly one unit, and every output element is
 * stored exactly once.  Word layout, for the problems with m, n, k >= 1 in
 * the caller's order, tiles of each problem in row-major tile order (before
 * rasterisation), k-blocks of tile_k:
 *   [0, total_iters)  word  iter_base(p) + tile * iters(p) + k_block
 *   then per global tile (tiles of all problems concatenated),
 *   (tile_m / 32) * (tile_n / 32) words, one per 32 x 32 block of the tile
 *   (block = (row / 32) * (tile_n / 32) + col / 32 within the tile).
 * Each visit adds SK_COVERAGE_VISIT(unit) (unit = CTA, or CTA pair when
 * tile_m == 256): after a correct call every word equals
 * SK_COVERAGE_VISIT(u) for one unit u, so (word & 0xff) counts the visits
 * and (word >> 8) - 1 names the unit. */
#define SK_COVERAGE_VISIT(unit) (1u + (((uint32_t)(unit) + 1u) << 8))

/* Timeline trace layout: CTA c owns entries [c*SK_TRACE_ENTRIES,
 * (c+1)*SK_TRACE_ENTRIES), each two uint64: (event << 32 | item index) and
 * %globaltimer in ns.  Entries 0..47 are written by the MMA issuer, 48..111
 * by the epilogue, 112..115 by the roles' lead threads, 116..121 by the
 * epilogue's fixup/spill/split detail, 122 at kernel entry; unused entries keep
 * the caller's contents (zero the buffer first). */
#define SK_TRACE_ENTRIES 128
#define SK_TRACE_BYTES_PER_CTA (SK_TRACE_ENTRIES * 16)
enum {
    SK_EV_START = 1,       /* CTA initialised (barriers, TMEM) */
    SK_EV_MMA_BEGIN = 2,   /* item: accumulator free, MMAs about to start */
    SK_EV_MMA_END = 4,     /* item: last MMA issued and committed */
    SK_EV_EPI_BEGIN = 5,   /* item: accumulator complete, epilogue starts */
    SK_EV_EPI_FLAGS = 6,   /* item (owner): every peer flag seen; split
                              reduce: every contributor has arrived */
    SK_EV_EPI_END = 7,     /* item: epilogue done (stores issued / flag raised) */
    SK_EV_END = 8,         /* a role is done (item = 0 producer, 1 MMA issuer,
                              2 epilogue); the CTA ends at the latest of them */
    SK_EV_ENTRY = 9,       /* the CTA entered the kernel (before any set-up) */
    SK_EV_FIX_ISSUE = 11,  /* last-item fixup: partial copies issued */
    SK_EV_FIX_FIRST = 12,  /*   first staged partial chunk arrived */
    SK_EV_FIX_LAST = 13,   /*   last chunk of the first batch arrived */
    SK_EV_SPILL_ISSUED = 14,  /* peer: partial stores issued */
    SK_EV_SPILL_VISIBLE = 15, /* peer (and split-reduce contributor): partial
                                 stores visible (after the fence) */
    SK_EV_SPLIT_SUMMED = 16   /* split reduce: this CTA's share summed and its
                                 C stores issued */
};

/* Resolved plan of a call, for inspection and tests. */
typedef struct {
    int tile_m, tile_n, tile_k, stages;
    sk_mode mode;            /* never AUTO */
    int num_ctas;            /* scheduler units g: CTAs, or CTA pairs if tile_m == 256 */
    int sk_units;            /* units that take Stream-K iterations */
    int64_t tiles;           /* output tiles over all problems */
    int64_t sk_tiles;        /* leading tiles computed Stream-K */
    int64_t dp_tiles;        /* tiles computed whole, round-robin */
    int64_t sk_iters;        /* k-block iterations of the Stream-K tiles */
    int64_t iters_per_unit;  /* floor(sk_iters / sk_units) */
    int64_t extra_units;     /* sk_iters mod sk_units: units with one more */
    size_t workspace_bytes;
    double predicted_us;     /* the library's runtime-model estimate of the call */
    sk_fixup fixup;          /* the fixup protocol the call uses */
    int64_t coverage_words;  /* uint32 words a sk_config.coverage buffer needs */
} sk_plan_info;

/* One unit of work of one CTA, in the order that CTA processes it. */
typedef enum { SK_ROLE_WHOLE = 0, SK_ROLE_OWNER = 1, SK_ROLE_PEER = 2, SK_ROLE_DP = 3 } sk_role;
typedef struct {
    int32_t problem;         /* index into the problem array */
    int32_t tile;            /* tile index within the problem, before rasterisation */
    int32_t tile_row, tile_col;   /* tile coordinates (rows of tile_m, cols of tile_n) */
    int32_t k0, k1;          /* k-block range [k0, k1) */
    int32_t role;            /* sk_role */
    int32_t peer_first;      /* OWNER: peers are CTAs peer_first..peer_last, */
    int32_t peer_last;       /*        added in this ascending order          */
    int32_t pad;
    int64_t global_tile;     /* tile index over the concatenated problems */
} sk_work_item;

/* Bytes of workspace a call with these problems and config needs
 * (per-CTA partial slots, per-CTA flags, one status word).  `count` >= 1.
 * If cfg->num_ctas is 0 the current device's SM count is used (needs a
 * device).  Host-only; no launch. */
SK_API sk_status sk_workspace_size(const sk_problem *problems, int count,
                            const sk_config *cfg, size_t *bytes);

/* Zero a workspace (flags and status word must start at zero).  Needed once
 * after allocation and after any call that reported SK_ERR_TIMEOUT; a
 * completed call leaves every flag it used back at zero. */
SK_API sk_status sk_workspace_init(void *ws, size_t ws_bytes, sk_stream_t stream);

/* C = alpha*A*B + beta*C_in for one problem.  ws must hold
 * sk_workspace_size() bytes, be 256-byte aligned, and not be used by
 * another call that may run concurrently on the GPU. */
SK_API sk_status sk_gemm(const sk_problem *problem, const sk_config *cfg,
                  void *ws, size_t ws_bytes, sk_stream_t stream);

/* `count` independent GEMMs (1 <= count <= 65536) in ONE persistent
 * launch.  The problems' tiles are concatenated and the decomposition runs
 * over all of them, so Stream-K ranges cross problem boundaries.  All
 * problems must share a_type, b_type and c_type (E4M3: one problem per
 * call).  Outputs must not overlap.  Up to 64 problems travel in the
 * kernel's parameter block; a larger group keeps its problem table (two
 * TMA descriptors and the shape of each problem) in the workspace, which
 * sk_workspace_size then sizes for it, and the call first writes the table
 * with small copy kernels on `stream` (one per 30 KB of table, each
 * carrying its bytes in its parameter block, so a captured CUDA graph
 * replays them too). */
SK_API sk_status sk_gemm_grouped(const sk_problem *problems, int count,
                          const sk_config *cfg, void *ws, size_t ws_bytes,
                          sk_stream_t stream);

/* Backward of C = A*B (alpha = 1 semantics): given dC (m x n, row-major,
 * leading dimension lddc, type fwd->c_type), compute
 *     dA = dC * B^T   (m x k, same type/layout as A, leading dimension ldda)
 *     dB = A^T * dC   (k x n, same type/layout as B, leading dimension lddb)
 * in one grouped launch of two Stream-K GEMMs.  Either of dA, dB may be
 * NULL to skip it.  BF16 only.  An operand these GEMMs would read MN-major
 * (a forward K-major operand, and dC for dB) is first copied to K-major
 * layout in the workspace, past the GEMMs' own bytes, when ws_bytes holds
 * sk_gemm_backward_workspace_size(); with a smaller workspace (at least
 * sk_workspace_size of the two GEMMs) they read the operands in place,
 * about 1.4x slower.  The result is the same either way: a copy changes no
 * value and the GEMMs' summation order does not depend on the layout. */
SK_API sk_status sk_gemm_backward(const sk_problem *fwd, const void *dC, int64_t lddc,
                           void *dA, int64_t ldda, void *dB, int64_t lddb,
                           const sk_config *cfg, void *ws, size_t ws_bytes,
                           sk_stream_t stream);

/* Workspace bytes with which sk_gemm_backward (same fwd shape/layouts,
 * need_dA / need_dB = whether dA / dB is computed, same config) reads
 * K-major copies of its MN-major operands.  Pointers in fwd are ignored. */
SK_API sk_status sk_gemm_backward_workspace_size(const sk_problem *fwd, int need_dA, int need_dB,
                                                 const sk_config *cfg, size_t *bytes);

/* dst = transpose of src for 16-bit elements (BF16): src is rows x cols
 * row-major with leading dimension ld_src >= cols, dst cols x rows row-major
 * with ld_dst >= rows; device pointers, 2-byte aligned (16-byte aligned
 * pointers and leading dimensions that are multiples of 8 take the vector
 * path).  The kernel sk_gemm_backward uses for its K-major operand copies;
 * asynchronous on `stream`.  rows or cols == 0: nothing to do. */
SK_API sk_status sk_transpose16(const void *src, int64_t rows, int64_t cols, int64_t ld_src,
                                void *dst, int64_t ld_dst, sk_stream_t stream);

/* Per-tensor FP8 quantisation: scale = amax(|x|)/448 (1 if x == 0),
 * q = E4M3(x / scale) rounded to nearest even and saturated to +-448.
 * x: n float32 values; q: n bytes; scale_out: one float; amax_work: one
 * float of scratch.  All device pointers. */
SK_API sk_status sk_quantize_e4m3(const float *x, int64_t n, uint8_t *q,
                           float *scale_out, float *amax_work,
                           sk_stream_t stream);

/* Synchronise `stream`, read the workspace's status word (SK_OK or
 * SK_ERR_TIMEOUT) into *device_status, and clear it if `clear`. */
SK_API sk_status sk_get_status(const void *ws, size_t ws_bytes, sk_stream_t stream,
                        int clear, sk_status *device_status);

/* Human-readable name of a status code (static string). */
SK_API const char *sk_status_string(sk_status s);

/* Resolve a call's plan without launching anything.  num_sms > 0 overrides
 * the device's SM count (then no device is needed). */
SK_API sk_status sk_plan_query(const sk_problem *problems, int count,
                        const sk_config *cfg, int num_sms, sk_plan_info *out);

/* The work items CTA `unit` of that plan processes, in order, computed by
 * the same scheduler code the kernels run.  Writes at most `max_items`
 * items and the total count to *n_items. */
SK_API sk_status sk_plan_unit_items(const sk_problem *problems, int count,
                             const sk_config *cfg, int num_sms, int unit,
                             sk_work_item *items, int max_items, int *n_items);

/* Description of the last failure this thread saw inside the library
 * (the CUDA call and its error string), or "" if none.  Static per-thread
 * storage, valid until the thread's next call into the library. */
SK_API const char *sk_last_error(void);

/* sk_gemm for callers that cannot allocate device memory.  (The paper has
 * no counterpart; this is a library convenience.)
 *
 * Who needs it: code whose device memory is owned entirely by another
 * allocator -- a framework's caching allocator or a pre-reserved memory
 * pool -- must not call cudaMalloc (it may synchronise the device and can
 * fail once the pool holds the memory), and plug-in style callers may have
 * nowhere to keep a workspace between calls.  This call needs neither: the
 * workspace is a fixed 12 MiB array inside the library, present on every
 * GPU that loads it until the process exits.  The call itself allocates
 * nothing (no cudaMalloc, cudaFree or allocating library routine).
 *
 * Same operands, config and result as sk_gemm, except that tile_n = 0
 * selects 128 here (so every SM fits).  Limit: the plan's workspace must
 * fit in 12 MiB -- 128x128 tiles on up to 191 CTAs, or 128x256 tiles on up
 * to 95 CTAs; the last-arriver fixup needs two partial slots per CTA, so
 * there 128x128 tiles on up to 95 CTAs.  Larger requests return
 * SK_ERR_WORKSPACE_TOO_SMALL before anything is launched.
 *
 * All calls share the one array per GPU.  Each call first zeroes the
 * array's flag region on `stream`, so calls ordered on the GPU are
 * independent, but calls that overlap on the GPU (different streams, no
 * ordering between them) race on the array and give undefined results.
 * The first call on a device (of this function or of sk_static_ws_status)
 * looks up the array's device address (once per device, with that device
 * current); make that first call before capturing any stream.  A device
 * wait that expires is recorded in the array's status word, which stays
 * set across later calls until sk_static_ws_status clears it. */
SK_API sk_status sk_gemm_static_ws(const sk_problem *problem, const sk_config *cfg,
                                   sk_stream_t stream);

/* The device-side status of sk_gemm_static_ws calls on the current device:
 * synchronise `stream`, read the fixed array's status word (SK_OK, or
 * SK_ERR_TIMEOUT if a bounded wait of any call since the last clear
 * expired) into *device_status, and clear it if `clear`.  (The paper has no
 * counterpart.)  Allocates nothing. */
SK_API sk_status sk_static_ws_status(sk_stream_t stream, int clear, sk_status *device_status);

/* Library version string. */
SK_API const char *sk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SKGEMM_H */
