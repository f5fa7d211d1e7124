/*
 * zf.h -- C ABI of the compressed-column transfer-and-decode library (libzf.so).
 *
 * The library implements the data path of ZipFlow (arXiv 2602.08190):
 * columns are compressed on the host and kept in pinned host memory
 * (Section 3, Fig. 3), their chunks are copied host-to-device and decoded on
 * the GPU, with copies of later chunks overlapping the decode of earlier ones
 * (Section 3.3, Pipelining Layer).  Decoders follow the three parallel
 * patterns of Section 3.1:
 *   Fully-Parallel  -- FOR + bit-packing, dictionary + bit-packing, raw
 *   Group-Parallel  -- delta + bit-packing (block prefix scan), run-length
 *   Non-Parallel    -- LZ77 byte blocks, one warp per block
 *
 * Conventions for every call:
 *   - Every function returns zf_status; ZF_OK (0) is success.  No call
 *     aborts, asserts or traps.  zf_last_error() describes the last failure
 *     seen by a context.
 *   - "host" pointers are CPU addresses; "device" pointers are CUDA device
 *     addresses on the context's device.
 *   - Objects created by the library (zf_ctx, zf_compressed, zf_resident) are
 *     owned by the caller once returned and are released with the matching
 *     *_destroy / *_free call.  Raw input columns and device output buffers
 *     stay owned by the caller; the library never keeps a pointer to them
 *     after the call that used them returns (zf_transfer_decompress keeps the
 *     output pointers until the matching zf_sync).
 *
 * Container format v1 (little-endian; produced by zf_compress_host,
 * accepted by zf_compressed_from_bytes):
 *   column = 64-byte column header | n_chunks x 32-byte directory | chunk blobs
 *     header: u32 magic 'ZCOL' | u16 version=1 | u8 scheme | u8 dtype |
 *             u32 n_chunks | u32 chunk_rows | u64 n_rows | u64 raw_bytes |
 *             u64 total_bytes | u32 flags (bit0: an int32 offsets column
 *             follows this BYTES column) | 20 zero bytes
 *     directory entry: u64 blob offset | u64 blob bytes | u64 first row |
 *             u32 rows | u32 0
 *   chunk blob = 64-byte chunk header | up to 3 sections | zero padding;
 *     every section starts on a 16-byte boundary, blob size is a multiple of 16.
 *     header: u32 magic 'ZCHK' | u8 scheme | u8 dtype | u8 bit width b |
 *             u8 flags | u32 rows | u32 n_aux | i64 reference |
 *             u32 section offset[3] | u32 section length[3] | 16 zero bytes
 *   sections per scheme:
 *     RAW      s0 = values
 *     FOR_BP   s0 = bit-packed (x - reference), b = bits(max - min)
 *     DICT_BP  s0 = sorted distinct values (n_aux of them, <= 65536),
 *              s1 = bit-packed ranks, b = bits(n_aux - 1)
 *     DELTA_BP s0 = n_aux 24-byte block entries {i64 base, i64 min_d,
 *              u32 payload offset in s1, u8 b, 3 zero bytes}, one per 1024
 *              rows; s1 = per block ceil(m*b/8) bytes padded to 16 of
 *              u_0 = 0, u_j = x_j - x_{j-1} - min_d
 *     RLE      s0 = run values, s1 = u32 run lengths (n_aux runs),
 *              s2 = one {u32 run, u32 rows of that run before} entry per
 *              1024 rows (the run holding row 1024*t)
 *     LZ77     rows = raw bytes of one block, n_aux = tokens T; flags bit0 =
 *              stored raw (s0).  Otherwise s0 = 2T-1 LEB128 lengths (each at
 *              most 3 bytes): literal length of token t at index 2t, match
 *              length - 4 of token t at 2t+1; s1 = T-1 u16 offsets (1..65535);
 *              s2 = literal bytes.  Token t copies its literals, then (all but
 *              the last token) `length` bytes from `offset` bytes back
 *     FLOAT2INT (F64 only) header byte 48 = decimal exponent e (0..18);
 *              s0 = bit-packed (d - reference), b = bits(max - min), of the
 *              integers d with v = d / 10^e; s1 = u32 rows of the n_aux
 *              exceptions (ascending), s2 = their 64-bit patterns.  The value
 *              of d is the double nearest d / 10^e; every d of a valid chunk
 *              has |d| <= 2^53 (decoders report larger ones as corrupt).
 *              Exception rows hold u = 0 in s0.
 *     STRDICT  (BYTES only; chunk_rows = bytes per chunk, a multiple of 65536,
 *              at most 2^26) rows = bytes of the chunk, n_aux = dictionary
 *              entries (1..65536), reference = tokens T, b = bits(n_aux - 1).
 *              s0 = u32 offsets of the n_aux + 1 entries in s1 (0, increasing,
 *              each entry 1..64 bytes, the last = s1's length), then u32 output
 *              offset of token 1024*j for j < ceil(T/1024); s1 = the entries'
 *              bytes; s2 = bit-packed entry numbers of the T tokens.  The chunk
 *              is the entries of the tokens, one after another.  The encoder
 *              cuts a token after each space byte, before each row start, after
 *              64 bytes and at the chunk end, sorts the distinct tokens by
 *              their bytes (a prefix first), and above 65536 distinct tokens
 *              makes every byte a token
 *     ANS      (I32/I64) header byte 48 = k (5..12): every 2^k rows form an
 *              independent stream; n_aux = distinct values (1..256),
 *              reference = streams K = ceil(rows/2^k), b = 12.  s0 = the sorted values;
 *              s1 = u16 frequency of each value (>= 1, summing to M = 4096;
 *              padded to 4 bytes), then u32 start of each stream in s2 and
 *              the end of the last; s2 = the streams.  Stream j holds rows
 *              j*2^k.. as range ANS: a u32 state x, then bytes; per row the
 *              value is the one whose [cumulative, cumulative + frequency)
 *              holds x mod M, x becomes f * (x / M) + x mod M - cumulative,
 *              and while x < 2^23 the next byte enters as x = 256 x + byte.
 *              A stream ends at x = 2^23 with every byte read
 *   Bit-packing: value i occupies stream bits [i*b, i*b+b), least
 *   significant bit first; stream bit k is bit k%8 of byte k/8.
 */
#ifndef ZF_H
#define ZF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    ZF_OK = 0,
    ZF_EINVAL = 1,        /* bad argument, unsupported scheme/dtype pair, call out of order */
    ZF_ENOMEM = 2,        /* host, pinned or device allocation failed */
    ZF_ECUDA = 3,         /* a CUDA runtime call failed */
    ZF_ECORRUPT = 4,      /* a compressed stream is malformed (host check or device decoder) */
    ZF_ETIMEOUT = 5,      /* reserved for a bounded device wait that gives up; no decoder of this
                             build waits (the batched work queue only counts), so none raises it */
    ZF_EUNSUPPORTED = 6,  /* feature not available in this build */
    ZF_EBUSY = 7          /* a transfer is in flight: call zf_sync first */
} zf_status;

typedef enum { ZF_I32 = 0, ZF_I64 = 1, ZF_BYTES = 2, ZF_F64 = 3 } zf_dtype;

typedef enum {
    ZF_RAW = 0, ZF_FOR_BP = 1, ZF_DICT_BP = 2, ZF_DELTA_BP = 3, ZF_RLE = 4, ZF_LZ77 = 5,
    ZF_FLOAT2INT = 6,     /* float64 columns (Section 2.1 "Float2Int", with bit-packing as in Table 2) */
    ZF_STRDICT = 7,       /* byte columns: dictionary of tokens + bit-packed codes (Section 2.1; Section 5.3.1) */
    ZF_ANS = 8,           /* integer columns of at most 256 values per chunk: dictionary + range ANS (Section 2.1) */
    ZF_NSCHEMES = 9
} zf_scheme;

typedef struct zf_ctx zf_ctx;
typedef struct zf_compressed zf_compressed;
typedef struct zf_resident zf_resident;

/* A raw column in host memory.  I32/I64/F64: `data` holds n values.  BYTES:
 * `data` holds offsets[n] bytes and `offsets` (host, int32) holds n+1
 * non-decreasing offsets with offsets[0] == 0. */
typedef struct {
    int32_t dtype;            /* zf_dtype */
    const void* data;
    uint64_t n;
    const int32_t* offsets;   /* BYTES only, else NULL */
} zf_column;

/* Kernel geometry, the <L,S,C> vector of Section 4: S = threads per CTA,
 * C = values a lane stores per 16-byte store (16 / value size), L = the
 * warp job's 1024-row tiles: each warp decodes tile_rows / 1024 consecutive
 * tiles of one chunk, staging the next tile while it decodes the current
 * one.  Zero fields take the built-in values. */
typedef struct {
    uint32_t tile_rows;       /* rows per warp job: a multiple of 1024, <= 16384 (0 = the
                                 class's tuned value, else 2048 for delta launches
                                 and 4096 for the others) */
    uint32_t threads;         /* 128, 256 or 512 (0 = the class's tuned value, else 128) */
    uint32_t ctas_per_sm;     /* batched launch: persistent grid = ctas_per_sm x SM count (0 = occupancy limit) */
    uint32_t stage_bytes;     /* pipeline stage: compressed bytes per H2D copy + decode step (default 64 MiB) */
    uint32_t flags;           /* ZF_KCFG_BATCHED: one work-queue launch per stage for the chunks of
                                 every Fully- and Group-Parallel scheme (LZ77 and ANS chunks keep
                                 their own kernels); else one launch per (scheme, dtype) group;
                                 ZF_KCFG_GRAPH: capture repeated transfers in a CUDA graph;
                                 ZF_KCFG_KEEP_ORDER: copy columns in the order given */
} zf_kcfg;

#define ZF_KCFG_BATCHED 1u
#define ZF_KCFG_GRAPH 2u
#define ZF_KCFG_KEEP_ORDER 4u   /* transfers keep the caller's column order (no Johnson's rule) */

typedef struct {
    int32_t scheme;           /* zf_scheme, or -1 to let the selector choose */
    uint32_t chunk_rows;      /* rows per chunk (BYTES: bytes per LZ77 block, fixed 65536); 0 = default */
    int32_t selector;         /* 0 = forced/heuristic, 1 = learned MLP, 2 = exhaustive measurement */
    int32_t offsets_scheme;   /* BYTES: scheme of the offsets column (FOR_BP or DELTA_BP); -1 = DELTA_BP */
    uint32_t ans_stream_rows; /* ANS: rows per independent stream, a power of two 32..4096 (0 = 512);
                                 Section 5.2.3's chunk-size trade of ratio for throughput */
} zf_plan_opts;

typedef struct {
    int32_t scheme;           /* zf_scheme chosen */
    uint32_t chunk_rows;
    int32_t offsets_scheme;   /* BYTES columns */
    zf_kcfg kcfg;
    float predicted_ms;       /* selector's or autotuner's estimate, 0 if none */
    int32_t label;            /* selector class (scheme, chunk size), -1 if none */
    uint32_t ans_stream_rows; /* ANS: rows per stream (0 = 512) */
} zf_plan_t;

/* Per-call statistics filled by zf_sync. */
typedef struct {
    uint64_t raw_bytes;       /* decoded bytes delivered */
    uint64_t comp_bytes;      /* compressed bytes copied host-to-device */
    uint32_t n_chunks;
    uint32_t n_stages;
    uint32_t n_launches;      /* kernels launched by the call */
    uint32_t device_error;    /* zf_status bits raised by the decoders (0 = none) */
    float total_ms;           /* first copy enqueue to last decode completion (CUDA events) */
    float copy_ms;            /* sum of copy times */
    float decode_ms;          /* sum of decode-kernel times */
} zf_stats;

/* ---- context ------------------------------------------------------------ */

/* Create a context on `device`.  `copy_stream` / `compute_stream` are
 * cudaStream_t handles (for example torch.cuda.Stream.cuda_stream) or NULL
 * to let the context create its own non-blocking streams.  The context owns
 * the staging ring, events, descriptor buffers and the device error word.
 * Calls on a context (and on a zf_mlp) work on its device and put the
 * calling thread's current device back before they return. */
zf_status zf_ctx_create(int device, void* copy_stream, void* compute_stream, zf_ctx** out);
zf_status zf_ctx_destroy(zf_ctx* ctx);
const char* zf_last_error(const zf_ctx* ctx);
/* Override the kernel geometry used when a plan does not carry one. */
zf_status zf_ctx_set_kcfg(zf_ctx* ctx, const zf_kcfg* kcfg);
/* Number of staging slots (2..8, default 8) and bytes per slot (0 = sized per call).
 * Each slot has its own decode stream, so up to `slots` stages decode at once. */
zf_status zf_ctx_set_ring(zf_ctx* ctx, uint32_t slots, uint64_t slot_bytes);

/* ---- planning and host compression (Section 3, offline path) ------------ */

/* Choose scheme, chunk size and kernel geometry for a column.  With
 * opts->scheme >= 0 the scheme is forced; otherwise opts->selector picks the
 * heuristic (0), the learned MLP (1, needs zf_ctx_set_selector) or exhaustive
 * measurement on the GPU (2).  F64 columns take FLOAT2INT (or a forced RAW):
 * the selector's classes cover integer and byte columns only.  `opts` may
 * be NULL. */
zf_status zf_plan(zf_ctx* ctx, const zf_column* col, const zf_plan_opts* opts, zf_plan_t* out);

/* Compress a host column with a plan into pinned host memory owned by the
 * returned object.  Runs on the CPU (threads over chunks).  Returns
 * ZF_EINVAL for a scheme that does not fit the column (for example a
 * dictionary above 65,536 entries) and ZF_ENOMEM if pinned memory runs out. */
zf_status zf_compress_host(const zf_plan_t* plan, const zf_column* col, zf_compressed** out);
zf_status zf_compressed_info(const zf_compressed* c, uint64_t* raw_bytes, uint64_t* comp_bytes, uint32_t* n_chunks);
zf_status zf_compressed_free(zf_compressed* c);
/* Serialized bytes of a compressed column (format above): *data points into
 * the object's pinned buffer and stays valid until zf_compressed_free. */
zf_status zf_compressed_bytes(const zf_compressed* c, const uint8_t** data, uint64_t* len);
/* Build a compressed object from serialized bytes (copied into pinned
 * memory).  The structure is validated on the host; ZF_ECORRUPT if not. */
zf_status zf_compressed_from_bytes(const uint8_t* data, uint64_t len, zf_compressed** out);

/* ---- transfer + decode (Section 3.3) ------------------------------------ */

/* Enqueue, for every column, the host-to-device copies of its chunks into
 * the staging ring (copy stream) and their decode into the caller's device
 * buffers (one decode stream per staging slot, joined into the compute
 * stream at the end).  Asynchronous: returns once enqueued.  Only the
 * context's streams are used: work of other streams on the output buffers
 * must be finished (or ordered before the copy stream with an event) by the
 * caller, and the outputs are complete once zf_sync returns.  d_out has
 * one device buffer per I32/I64 column and two per BYTES column (bytes,
 * then int32 offsets); d_out_bytes gives each buffer's capacity.  Returns
 * ZF_EBUSY if the previous call was not synced. */
zf_status zf_transfer_decompress(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes);
/* Wait for the last transfer (or resident decode) to finish.  Returns the
 * first host-side error, else ZF_ECORRUPT raised by the decoders.
 * `stats` may be NULL. */
zf_status zf_sync(zf_ctx* ctx, zf_stats* stats);

/* Columns of a transfer are copied in the order of Johnson's rule for the
 * two-stage flow (copy, then decode) of Section 3.3: columns whose copy is
 * shorter than their decode first, by increasing copy time, then the rest by
 * decreasing decode time (minimum makespan of the two-machine flow shop).  A
 * column's copy time is its compressed bytes over the link rate last measured
 * by zf_measure_copy on the context (200 GB/s before any), its decode time
 * each chunk's plain bytes over the decode rate zf_tune measured for the
 * chunk's (scheme, dtype, bit-width bucket) class (a nominal rate per scheme
 * before any).  ZF_KCFG_KEEP_ORDER turns the reordering off. */

/* The order Johnson's rule gives n jobs with times copy_ms[i] (first stage)
 * and decode_ms[i] (second stage): order[] receives a permutation of 0..n-1
 * (host arrays; ties keep the input order).  ZF_EINVAL for a negative or NaN
 * time.  This is the ordering zf_transfer_decompress applies to columns. */
zf_status zf_johnson_order(const float* copy_ms, const float* decode_ms, uint32_t n, uint32_t* order);

/* The raw link at a call's own piece sizes: copy the columns' compressed
 * bytes host-to-device exactly as zf_transfer_decompress would stage them
 * (same stages, same 128-byte aligned pieces, same staging slots and copy
 * stream) without decoding, `reps` times after one warm-up (0 = 5).  *ms =
 * the fastest run (CUDA events on the copy stream).  The rate (compressed
 * bytes / *ms) is kept by the context for Johnson's rule.  Returns ZF_EBUSY
 * while a transfer is in flight. */
zf_status zf_measure_copy(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols, uint32_t reps, float* ms);

/* Copy a compressed column into device memory once, for decoding with the
 * compressed bytes already resident in HBM. */
zf_status zf_upload(zf_ctx* ctx, const zf_compressed* c, zf_resident** out);
zf_status zf_resident_free(zf_resident* r);
/* Enqueue the decode of resident columns on the compute stream
 * (asynchronous; finish with zf_sync).  Outputs as in zf_transfer_decompress. */
zf_status zf_decompress_resident(zf_ctx* ctx, const zf_resident* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes);

/* ---- autotuning (Section 4, device geometry; Section 5.5) ------------------ */

/* One measured point of the search: the geometry and its median time. */
typedef struct {
    zf_kcfg kcfg;
    float ms;                 /* median of `reps` runs: zf_stats.total_ms (resident) or host wall clock (transfer) */
} zf_tune_point;

/* Exhaustive search of the kernel geometry for these columns, the
 * brute-force search of Section 5.5 on this GPU: every tile_rows in
 * {1024, 2048, 4096, 8192, 16384} (L = 1..16 tiles per warp job) x threads in
 * {128, 256, 512} (S) is run once to warm up and `reps` times (0 = 3); with
 * `transfer` != 0 the full transfer is timed and stage_bytes in
 * {4, 8, 16, 32, 64} MiB and graph replay (ZF_KCFG_GRAPH off, then on) are
 * searched too (150 points, each timed on the host clock around the call and
 * zf_sync, as a caller sees it), otherwise the decode of the columns uploaded
 * to HBM (15 points, timed by device events).  C is fixed by the store width.
 * Writes up to max_points points (every point is visited once, in that
 * order), sets *n_points to the number visited and stores the fastest
 * geometry in *best (nullable).  When all chunks of the columns are of one
 * class -- the same scheme, dtype and bit-width bucket (widest b <= 8, 16,
 * 32, 64; for string columns the class of their bytes, the offsets being a
 * small second part) -- the result is kept for that class: later launches of the class
 * use it while the context's tile_rows / threads are 0 (automatic), so one
 * tuning run per column kind gives every kind its own geometry.  Otherwise
 * the result becomes the context's geometry.  A resident search of one
 * class also records the class's decode rate at the fastest point (plain
 * bytes / time), which Johnson's rule then uses.  Outputs as in
 * zf_transfer_decompress; the columns are decoded into them many times. */
zf_status zf_tune(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols, void* const* d_out,
                  const uint64_t* d_out_bytes, int32_t transfer, uint32_t reps, zf_tune_point* points,
                  uint32_t max_points, uint32_t* n_points, zf_kcfg* best);

/* The chunk-size dimension of the search (the C of Section 4's <L,S,C> plus
 * the chunk size the transfer moves): encode the host column `col` with
 * `scheme` at each of the n candidate chunk sizes chunk_rows[i] (rows per
 * chunk; bytes per chunk for a string dictionary), time the transfer +
 * decode of each (`reps` runs after one warm-up, 0 = 3; median of zf_sync's
 * total_ms) into ms[i], -1 where the scheme or size does not fit the column,
 * and set *best (nullable) to the index of the fastest.  ZF_EINVAL if none
 * fits.  The context's geometry and ring are used as they are. */
zf_status zf_tune_chunk_rows(zf_ctx* ctx, const zf_column* col, int32_t scheme, const uint32_t* chunk_rows,
                             uint32_t n, uint32_t reps, float* ms, uint32_t* best);

/* The geometry a launch of one class would use now: the context's
 * tile_rows / threads where set, else the class's tuned entry, else the
 * built-in values (128 threads; warp jobs of 2048 rows for delta, 4096 for
 * the others).  bmax = the widest bit width of the launch's chunks. */
zf_status zf_ctx_tuned_geometry(const zf_ctx* ctx, int32_t scheme, int32_t dtype, uint32_t bmax, zf_kcfg* out);

/* The measured rates Johnson's rule reads for a class: the decode rate a
 * resident zf_tune of that class recorded (plain GB/s) and the link rate the
 * last zf_measure_copy recorded (compressed GB/s); 0 where none was measured
 * (the ordering then uses nominal rates).  Either pointer may be NULL. */
zf_status zf_ctx_rates(const zf_ctx* ctx, int32_t scheme, int32_t dtype, uint32_t bmax, float* decode_gbs,
                       float* link_gbs);

/* ---- learned selector ------------------------------------------------------ */

/* The 32 statistics of a host column the selector reads (value range,
 * distinct values, runs, differences, entropies, byte repetition ...),
 * each scaled to about [0, 1], computed on a fixed sample of the column:
 * the whole column up to 262,144 rows (bytes for string columns), else 64
 * windows of 4,096 consecutive rows.  out: 32 floats (host). */
zf_status zf_column_features(const zf_column* col, float* out);

/* A perceptron 32 -> 64 -> 64 -> 12 (ReLU, FP32) on a device, trained and run
 * by the library's CUDA kernels.  Classes: label = scheme * 2 + size, size 0
 * = 4 MiB and 1 = 32 MiB of uncompressed bytes per chunk.  Parameters are
 * 7,052 floats: W1[64][32], b1[64], W2[64][64], b2[64], W3[12][64], b3[12]. */
typedef struct zf_mlp zf_mlp;
#define ZF_MLP_PARAMS 7052
#define ZF_MLP_CLASSES 12
/* He-normal weights from `seed`, zero biases, Adam state cleared. */
zf_status zf_mlp_create(int device, uint64_t seed, zf_mlp** out);
zf_status zf_mlp_destroy(zf_mlp* net);
/* Copy the parameters out (host, 7,052 floats) or in (also clears Adam state
 * and the fitted input scaling). */
zf_status zf_mlp_get_params(const zf_mlp* net, float* host);
zf_status zf_mlp_set_params(zf_mlp* net, const float* host);
/* Device buffers: d_x batch x 32, d_logits batch x 12, d_y batch labels,
 * d_mask batch x 12 bytes (1 = class allowed), d_grad 7,052 floats, d_loss
 * one float (nullable).  `stream` is a cudaStream_t or NULL. */
zf_status zf_mlp_forward(zf_mlp* net, const float* d_x, uint32_t batch, float* d_logits, void* stream);
/* Gradient of the mean masked softmax cross-entropy of the batch. */
zf_status zf_mlp_grad(zf_mlp* net, const float* d_x, const int32_t* d_y, const uint8_t* d_mask, uint32_t batch,
                      float* d_grad, float* d_loss, void* stream);
/* One Adam step (b1 0.9, b2 0.999, eps 1e-8) with learning rate lr. */
zf_status zf_mlp_adam(zf_mlp* net, const float* d_grad, float lr, void* stream);
/* Train on host arrays (count samples): `epochs` passes in seeded random
 * order, mini-batches of `batch`, Adam at lr.  h_losses (nullable) gets the
 * mean loss of each epoch.  The inputs are standardized as (x - mean) / std
 * per feature, with the mean and standard deviation of these rows (std 1 for
 * a constant feature); the network keeps them and zf_mlp_predict and the
 * learned selector of zf_plan apply them (zf_mlp_get_scaling reads them). */
zf_status zf_mlp_train(zf_mlp* net, const float* h_x, const int32_t* h_y, const uint8_t* h_mask, uint32_t count,
                       uint32_t epochs, uint32_t batch, float lr, uint64_t seed, float* h_losses);
/* Class of each host row (argmax of the logits over its allowed classes, -1
 * if none allowed), computed on the GPU; rows are standardized first with the
 * scaling zf_mlp_train fitted (none after zf_mlp_set_params). */
zf_status zf_mlp_predict(zf_mlp* net, const float* h_x, const uint8_t* h_mask, uint32_t count, int32_t* h_class);
/* Time every selector class on a column: compress with the class's scheme
 * and chunk size, then transfer + decode (reps runs after one warm-up, median
 * of zf_sync's total_ms).  ms: 12 floats, -1 for classes that do not apply.
 * This is the exhaustive search zf_plan's selector 2 uses and the label
 * source for training the selector. */
zf_status zf_measure_classes(zf_ctx* ctx, const zf_column* col, uint32_t reps, float* ms);
/* Use `net` (kept, not owned) for zf_plan's selector 1.  With mean and std
 * NULL the features go through the scaling the network fitted in
 * zf_mlp_train; given (32-float host vectors, for a network loaded with
 * zf_mlp_set_params) they are standardized as (f - mean) / std instead. */
zf_status zf_ctx_set_selector(zf_ctx* ctx, zf_mlp* net, const float* mean, const float* std);
/* The input scaling the network fitted (mean 0, std 1 if none): 32 floats each. */
zf_status zf_mlp_get_scaling(const zf_mlp* net, float* mean, float* std);

/* ---- decode without allocation ------------------------------------------ */

/* Decode one compressed I32/I64 column (scheme RAW, FOR_BP, DICT_BP,
 * DELTA_BP or RLE) or F64 column (RAW or FLOAT2INT) whose serialized bytes (the format above, for example
 * zf_compressed_bytes copied to the GPU) already sit in device memory at
 * `d_column`, into the device buffer `d_out`, on `stream` (a cudaStream_t,
 * or NULL for the default stream).  The paper has no counterpart: this entry
 * point exists for callers that may not allocate device memory once they are
 * running -- engines that reserve all device memory at start-up, code whose
 * memory budget belongs to another runtime, or code that must not grow the
 * device heap inside a call.  It calls no cudaMalloc, cudaFree or other
 * allocating routine and needs no zf_ctx.
 *
 * Its scratch (chunk descriptors, work-queue counters, error word) is one
 * fixed device array of 262,400 bytes in the library, held by every GPU
 * that loads the library until the process exits.  It fits columns of at
 * most 4096 chunks; larger columns return ZF_EINVAL before any GPU work.
 * The first call on a device looks up the array's device address, so make
 * that first call before any stream capture.  The call is synchronous: it
 * returns after the decode has finished and reports ZF_ECORRUPT if the
 * device checks of the stream failed.  Every call on a device shares the
 * array (each call rewrites what it uses); calls that overlap on the GPU,
 * from several host threads or streams at once, race -- serialize them.
 * Both pointers must be 16-byte aligned; `out_bytes` must hold all rows.
 * Returns ZF_EUNSUPPORTED for BYTES and ANS columns.  Besides the checks of the
 * other entry points' kernels, the device checks that each Float2Int chunk's
 * exception rows are strictly increasing and inside the chunk. */
zf_status zf_decompress_device_noalloc(const void* d_column, uint64_t column_bytes, void* d_out,
                                       uint64_t out_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ZF_H */
