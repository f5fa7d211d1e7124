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
 *     LZ77     rows = raw bytes of one block; flags bit0 = stored raw (s0);
 *              otherwise s0 = tokens, s1 = literals; a token is a LEB128
 *              literal length and, unless it is the last of the block, a u16
 *              offset (1..65535) and a LEB128 (match length - 4)
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
    ZF_ETIMEOUT = 5,      /* a bounded device wait gave up */
    ZF_EUNSUPPORTED = 6,  /* feature not available in this build */
    ZF_EBUSY = 7          /* a transfer is in flight: call zf_sync first */
} zf_status;

typedef enum { ZF_I32 = 0, ZF_I64 = 1, ZF_BYTES = 2 } zf_dtype;

typedef enum {
    ZF_RAW = 0, ZF_FOR_BP = 1, ZF_DICT_BP = 2, ZF_DELTA_BP = 3, ZF_RLE = 4, ZF_LZ77 = 5,
    ZF_NSCHEMES = 6
} zf_scheme;

typedef struct zf_ctx zf_ctx;
typedef struct zf_compressed zf_compressed;
typedef struct zf_resident zf_resident;

/* A raw column in host memory.  I32/I64: `data` holds n values.  BYTES:
 * `data` holds offsets[n] bytes and `offsets` (host, int32) holds n+1
 * non-decreasing offsets with offsets[0] == 0. */
typedef struct {
    int32_t dtype;            /* zf_dtype */
    const void* data;
    uint64_t n;
    const int32_t* offsets;   /* BYTES only, else NULL */
} zf_column;

/* Kernel geometry, the <L,S,C> vector of Section 4: S = threads per CTA,
 * C = values a thread handles per 16-byte store, L = tile_rows / (S*C)
 * loop iterations per tile.  Zero fields take the tuned or built-in value. */
typedef struct {
    uint32_t tile_rows;       /* rows per CTA tile: a multiple of 1024, <= 65536; raised to
                                 1024 x threads/32 (one 1024-row warp tile per warp) */
    uint32_t threads;         /* 128, 256 or 512 */
    uint32_t ctas_per_sm;     /* persistent grid = ctas_per_sm x SM count (0 = occupancy limit) */
    uint32_t stage_bytes;     /* pipeline stage: compressed bytes per H2D copy + decode step */
    uint32_t flags;           /* ZF_KCFG_BATCHED: one work-queue launch per stage for all schemes
                                 (else one launch per (scheme, dtype) group);
                                 ZF_KCFG_GRAPH: capture repeated transfers in a CUDA graph */
} zf_kcfg;

#define ZF_KCFG_BATCHED 1u
#define ZF_KCFG_GRAPH 2u

typedef struct {
    int32_t scheme;           /* zf_scheme, or -1 to let the selector choose */
    uint32_t chunk_rows;      /* rows per chunk (BYTES: bytes per LZ77 block, fixed 65536); 0 = default */
    int32_t selector;         /* 0 = forced/heuristic, 1 = learned MLP, 2 = exhaustive measurement */
    int32_t offsets_scheme;   /* BYTES: scheme of the offsets column (FOR_BP or DELTA_BP); -1 = DELTA_BP */
} zf_plan_opts;

typedef struct {
    int32_t scheme;           /* zf_scheme chosen */
    uint32_t chunk_rows;
    int32_t offsets_scheme;   /* BYTES columns */
    zf_kcfg kcfg;
    float predicted_ms;       /* selector's or autotuner's estimate, 0 if none */
    int32_t label;            /* selector class (scheme, chunk size), -1 if none */
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
 * the staging ring, events, descriptor buffers and the device error word. */
zf_status zf_ctx_create(int device, void* copy_stream, void* compute_stream, zf_ctx** out);
zf_status zf_ctx_destroy(zf_ctx* ctx);
const char* zf_last_error(const zf_ctx* ctx);
/* Override the kernel geometry used when a plan does not carry one. */
zf_status zf_ctx_set_kcfg(zf_ctx* ctx, const zf_kcfg* kcfg);
/* Number of staging slots (2..8, default 2) and bytes per slot (0 = sized per call). */
zf_status zf_ctx_set_ring(zf_ctx* ctx, uint32_t slots, uint64_t slot_bytes);

/* ---- planning and host compression (Section 3, offline path) ------------ */

/* Choose scheme, chunk size and kernel geometry for a column.  With
 * opts->scheme >= 0 the scheme is forced; otherwise opts->selector picks the
 * heuristic (0), the learned MLP (1, needs zf_selector_load) or exhaustive
 * measurement on the GPU (2).  `opts` may be NULL. */
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
 * buffers (compute stream).  Asynchronous: returns once enqueued.  d_out has
 * one device buffer per I32/I64 column and two per BYTES column (bytes,
 * then int32 offsets); d_out_bytes gives each buffer's capacity.  Returns
 * ZF_EBUSY if the previous call was not synced. */
zf_status zf_transfer_decompress(zf_ctx* ctx, const zf_compressed* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes);
/* Wait for the last transfer (or resident decode) to finish.  Returns the
 * first host-side error, else ZF_ECORRUPT / ZF_ETIMEOUT raised by the
 * decoders.  `stats` may be NULL. */
zf_status zf_sync(zf_ctx* ctx, zf_stats* stats);

/* Copy a compressed column into device memory once, for decoding with the
 * compressed bytes already resident in HBM. */
zf_status zf_upload(zf_ctx* ctx, const zf_compressed* c, zf_resident** out);
zf_status zf_resident_free(zf_resident* r);
/* Enqueue the decode of resident columns on the compute stream
 * (asynchronous; finish with zf_sync).  Outputs as in zf_transfer_decompress. */
zf_status zf_decompress_resident(zf_ctx* ctx, const zf_resident* const* cols, uint32_t ncols,
                                 void* const* d_out, const uint64_t* d_out_bytes);

/* ---- decode without allocation ------------------------------------------ */

/* Decode one compressed I32/I64 column (scheme RAW, FOR_BP, DICT_BP,
 * DELTA_BP or RLE) whose serialized bytes (the format above, for example
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
 * Returns ZF_EUNSUPPORTED for BYTES columns. */
zf_status zf_decompress_device_noalloc(const void* d_column, uint64_t column_bytes, void* d_out,
                                       uint64_t out_bytes, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ZF_H */
