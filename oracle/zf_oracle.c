/*
 * zf_oracle.c -- plain, slow CPU oracle for the compressed-column codecs.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or constant with the GPU library: it re-implements the
 * container format from its written description, and every codec from the
 * paper's definitions:
 *
 *   Bit-packing / Frame of Reference   Section 2.1 ("Bit-packing and FOR")
 *   Dictionary encoding                Section 2.1; Section 3.1, Fig. 6(a)
 *   Delta encoding                     Section 2.1 ("Delta encoding")
 *   Run-length encoding, presum        Section 2.1 ("RLE"); Section 3.2
 *   LZ77 back-references               Section 2.1 (LZ77-based algorithms)
 *   Float2Int (+ bit-packing)          Section 2.1 ("Float2Int"); Table 2
 *   String dictionary (+ bit-packing)  Section 2.1 (dictionary encoding); Section 5.3.1
 *                                      (the comment column's words as dictionary codes)
 *   Dictionary + ANS                   Section 2.1 (entropy-based algorithms, ANS);
 *                                      Section 3.1 (ANS decode as the Non-Parallel example);
 *                                      the rANS coder itself is Duda's published method
 *   Independent chunks                 Section 3.1 (Non-Parallel "file chunking")
 *
 * Decoders are the definitions written out: values are read bit by bit,
 * delta adds each difference to the previous value, RLE expands each run at
 * its presum, and LZ77 copies a back-reference byte by byte.
 *
 * Parity: every function here is pinned by the not-gpu tests (closed forms,
 * brute force, hand-worked byte examples, library routines on special cases).
 *
 * Container format v1 (little-endian):
 *   column  = 64-byte column header, n_chunks x 32-byte chunk directory, chunk blobs
 *   chunk   = 64-byte chunk header, up to three sections, each 16-byte aligned,
 *             zero padding, blob length a multiple of 16
 * The layout constants below are typed in from that description.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- status codes (values of the library's zf_status) ---- */
enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ECORRUPT = 4 };
/* ---- schemes and dtypes ---- */
enum { ORC_RAW = 0, ORC_FOR_BP = 1, ORC_DICT_BP = 2, ORC_DELTA_BP = 3, ORC_RLE = 4, ORC_LZ77 = 5, ORC_F2I = 6,
       ORC_STRDICT = 7, ORC_ANS = 8 };
enum { ORC_I32 = 0, ORC_I64 = 1, ORC_BYTES = 2, ORC_F64 = 3 };

#define COL_MAGIC 0x4C4F435Au   /* "ZCOL" */
#define CHK_MAGIC 0x4B48435Au   /* "ZCHK" */
#define DELTA_BLOCK 1024u
#define RLE_DIR_ROWS 1024u
#define LZ_HASH_BITS 14
#define LZ_MIN_MATCH 4u
#define LZ_MAX_OFFSET 65535u
#define STR_TOKEN_MAX 64u     /* bytes in one string-dictionary token at most */
#define STR_DICT_MAX 65536u   /* dictionary entries at most */
#define STR_TILE 1024u        /* tokens per tile-start entry */
#define ANS_SCALE 12u         /* frequencies sum to M = 2^12 */
#define ANS_M (1u << ANS_SCALE)
#define ANS_L (1u << 23)      /* states stay in [L, 256 L) */
#define ANS_LOG_MIN 5u        /* rows per independent stream: 2^5 .. 2^12, stored as log2 in header byte 48 */
#define ANS_LOG_MAX 12u
#define ANS_SUB_DEFAULT 512u  /* rows per stream when the caller names none */

/* ------------------------------------------------------------------------- */
/* little-endian byte helpers                                                */
/* ------------------------------------------------------------------------- */
static void put_u16(uint8_t* p, uint32_t v) { p[0] = (uint8_t)v; p[1] = (uint8_t)(v >> 8); }
static void put_u32(uint8_t* p, uint32_t v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static void put_u64(uint8_t* p, uint64_t v) { for (int i = 0; i < 8; i++) p[i] = (uint8_t)(v >> (8 * i)); }
static uint32_t get_u16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t get_u32(const uint8_t* p) { uint32_t v = 0; for (int i = 0; i < 4; i++) v |= (uint32_t)p[i] << (8 * i); return v; }
static uint64_t get_u64(const uint8_t* p) { uint64_t v = 0; for (int i = 0; i < 8; i++) v |= (uint64_t)p[i] << (8 * i); return v; }
static uint64_t align16(uint64_t x) { return (x + 15) / 16 * 16; }

/* number of bits needed for x: 0 for x == 0, else floor(log2 x) + 1 */
uint32_t orc_bits(uint64_t x) {
    uint32_t b = 0;
    while (x) { b++; x >>= 1; }
    return b;
}

static unsigned width_of(int dtype) { return dtype == ORC_I64 ? 64u : 32u; }
static unsigned size_of(int dtype) { return (dtype == ORC_I64 || dtype == ORC_F64) ? 8u : (dtype == ORC_I32 ? 4u : 1u); }
static uint64_t mask_of(unsigned w) { return w >= 64 ? ~0ull : ((1ull << w) - 1); }

/* value i of a typed array as a sign-extended 64-bit integer */
static int64_t load_val(const void* data, int dtype, uint64_t i) {
    if (dtype == ORC_I64) return ((const int64_t*)data)[i];
    return (int64_t)((const int32_t*)data)[i];
}
static void store_val(void* data, int dtype, uint64_t i, uint64_t v) {
    if (dtype == ORC_I64) ((int64_t*)data)[i] = (int64_t)v;
    else ((int32_t*)data)[i] = (int32_t)(uint32_t)v;
}
/* reinterpret the low w bits of v as a signed w-bit integer */
static int64_t sext(uint64_t v, unsigned w) {
    if (w >= 64) return (int64_t)v;
    v &= mask_of(w);
    if (v >> (w - 1)) return (int64_t)(v | ~mask_of(w));
    return (int64_t)v;
}

/* ------------------------------------------------------------------------- */
/* Bit-packing (Section 2.1): value i occupies stream bits [i*b, i*b+b),     */
/* least significant bit first; stream bit k is bit (k mod 8) of byte k/8.   */
/* ------------------------------------------------------------------------- */
uint64_t orc_packed_bytes(uint64_t n, uint32_t b) { return (n * (uint64_t)b + 7) / 8; }

/* writes exactly ceil(n*b/8) bytes; `out` must hold them and is overwritten */
uint64_t orc_pack(const uint64_t* u, uint64_t n, uint32_t b, uint8_t* out) {
    uint64_t nbytes = orc_packed_bytes(n, b);
    memset(out, 0, nbytes);
    for (uint64_t i = 0; i < n; i++)
        for (uint32_t k = 0; k < b; k++)
            if ((u[i] >> k) & 1ull) {
                uint64_t bit = i * b + k;
                out[bit / 8] |= (uint8_t)(1u << (bit % 8));
            }
    return nbytes;
}

uint64_t orc_unpack_one(const uint8_t* in, uint64_t i, uint32_t b) {
    uint64_t v = 0;
    for (uint32_t k = 0; k < b; k++) {
        uint64_t bit = i * b + k;
        if ((in[bit / 8] >> (bit % 8)) & 1u) v |= 1ull << k;
    }
    return v;
}

/* ------------------------------------------------------------------------- */
/* chunk assembly                                                            */
/* ------------------------------------------------------------------------- */
typedef struct {
    uint8_t* p;       /* chunk start */
    uint64_t end;     /* bytes used so far (relative to chunk start) */
} chunk_w;

/* start section s at the next 16-byte boundary; returns its offset */
static uint64_t sec_begin(chunk_w* w, int s, uint64_t len) {
    uint64_t off = align16(w->end);
    put_u32(w->p + 24 + 4 * s, (uint32_t)off);
    put_u32(w->p + 36 + 4 * s, (uint32_t)len);
    w->end = off + len;
    return off;
}

static void chunk_header(uint8_t* p, int scheme, int dtype, uint32_t bw, uint32_t flags,
                         uint32_t rows, uint32_t n_aux, uint64_t ref) {
    memset(p, 0, 64);
    put_u32(p + 0, CHK_MAGIC);
    p[4] = (uint8_t)scheme;
    p[5] = (uint8_t)dtype;
    p[6] = (uint8_t)bw;
    p[7] = (uint8_t)flags;
    put_u32(p + 8, rows);
    put_u32(p + 12, n_aux);
    put_u64(p + 16, ref);
}

/* upper bound of one chunk's blob */
static uint64_t chunk_bound(int scheme, int dtype, uint64_t rows) {
    uint64_t sz = size_of(dtype);
    uint64_t b = 64 + 3 * 16;
    switch (scheme) {
    case ORC_RAW: case ORC_FOR_BP: return b + rows * sz;
    case ORC_DICT_BP: return b + rows * sz + rows * 2 + 16;
    case ORC_DELTA_BP: return b + (rows / DELTA_BLOCK + 1) * (24 + 16) + rows * sz + 16;
    case ORC_RLE: return b + rows * (sz + 4) + (rows / RLE_DIR_ROWS + 1) * 8;
    case ORC_LZ77: return b + rows + rows / 2 + 64;
    case ORC_F2I: return b + rows * (8 + 4 + 8) + 32;
    case ORC_STRDICT: return b + 4 * (rows + 2 + rows / STR_TILE + 1) + rows + 2 * rows + 32;
    case ORC_ANS: return b + 256 * sz + 512 + 8 * (rows / (1u << ANS_LOG_MIN) + 2) + 2 * rows + 32;
    }
    return 0;
}

/* ---- RAW ---- */
static uint64_t enc_raw(uint8_t* p, int dtype, const void* x, uint32_t m) {
    chunk_w w = {p, 64};
    chunk_header(p, ORC_RAW, dtype, 0, 0, m, 0, 0);
    uint64_t off = sec_begin(&w, 0, (uint64_t)m * size_of(dtype));
    memcpy(p + off, x, (uint64_t)m * size_of(dtype));
    return align16(w.end);
}

/* ---- FOR + bit-packing: reference = chunk minimum, b from max - min ---- */
static uint64_t enc_for(uint8_t* p, int dtype, const void* x, uint32_t m) {
    unsigned w_ = width_of(dtype);
    int64_t mn = 0, mx = 0;
    for (uint32_t i = 0; i < m; i++) {
        int64_t v = load_val(x, dtype, i);
        if (i == 0 || v < mn) mn = v;
        if (i == 0 || v > mx) mx = v;
    }
    uint32_t b = orc_bits(((uint64_t)mx - (uint64_t)mn) & mask_of(w_));
    uint64_t* u = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    for (uint32_t i = 0; i < m; i++) u[i] = ((uint64_t)load_val(x, dtype, i) - (uint64_t)mn) & mask_of(w_);
    chunk_w w = {p, 64};
    chunk_header(p, ORC_FOR_BP, dtype, b, 0, m, 0, (uint64_t)mn);
    uint64_t off = sec_begin(&w, 0, orc_packed_bytes(m, b));
    orc_pack(u, m, b, p + off);
    free(u);
    return align16(w.end);
}

/* ---- dictionary: sorted distinct values, code = rank, bit-packed ---- */
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}
static uint64_t enc_dict(uint8_t* p, int dtype, const void* x, uint32_t m, int* err) {
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (m ? m : 1));
    for (uint32_t i = 0; i < m; i++) s[i] = load_val(x, dtype, i);
    qsort(s, m, sizeof(int64_t), cmp_i64);
    uint32_t nd = 0;
    for (uint32_t i = 0; i < m; i++)
        if (i == 0 || s[i] != s[nd - 1]) s[nd++] = s[i];
    if (nd > 65536) { free(s); *err = ORC_EINVAL; return 0; }
    uint32_t b = nd > 0 ? orc_bits(nd - 1) : 0;
    uint64_t* code = (uint64_t*)malloc(sizeof(uint64_t) * (m ? m : 1));
    for (uint32_t i = 0; i < m; i++) {
        int64_t v = load_val(x, dtype, i);
        uint32_t lo = 0, hi = nd;          /* lower bound of v in the dictionary */
        while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (s[mid] < v) lo = mid + 1; else hi = mid; }
        code[i] = lo;
    }
    chunk_w w = {p, 64};
    chunk_header(p, ORC_DICT_BP, dtype, b, 0, m, nd, 0);
    uint64_t doff = sec_begin(&w, 0, (uint64_t)nd * size_of(dtype));
    for (uint32_t k = 0; k < nd; k++) store_val(p + doff, dtype, k, (uint64_t)s[k]);
    uint64_t coff = sec_begin(&w, 1, orc_packed_bytes(m, b));
    orc_pack(code, m, b, p + coff);
    free(s); free(code);
    return align16(w.end);
}

/* ---- delta: per 1024-row block, base + differences (+ FOR on the differences) ---- */
static uint64_t enc_delta(uint8_t* p, int dtype, const void* x, uint32_t m) {
    unsigned wd = width_of(dtype);
    uint64_t msk = mask_of(wd);
    uint32_t nb = (m + DELTA_BLOCK - 1) / DELTA_BLOCK;
    chunk_w w = {p, 64};
    chunk_header(p, ORC_DELTA_BP, dtype, 0, 0, m, nb, 0);
    uint64_t toff = sec_begin(&w, 0, (uint64_t)nb * 24);
    /* first pass: widths, to size the payload section */
    uint64_t* u = (uint64_t*)malloc(sizeof(uint64_t) * DELTA_BLOCK);
    uint64_t payload_total = 0;
    for (int pass = 0; pass < 2; pass++) {
        uint64_t poff = 0, sec1 = 0;
        if (pass == 1) sec1 = sec_begin(&w, 1, payload_total);
        for (uint32_t k = 0; k < nb; k++) {
            uint32_t r0 = k * DELTA_BLOCK;
            uint32_t mk = m - r0 < DELTA_BLOCK ? m - r0 : DELTA_BLOCK;
            int64_t base = load_val(x, dtype, r0);
            int64_t min_d = 0;
            for (uint32_t j = 1; j < mk; j++) {
                int64_t d = sext((uint64_t)load_val(x, dtype, r0 + j) - (uint64_t)load_val(x, dtype, r0 + j - 1), wd);
                if (j == 1 || d < min_d) min_d = d;
            }
            uint64_t umax = 0;
            u[0] = 0;
            for (uint32_t j = 1; j < mk; j++) {
                int64_t d = sext((uint64_t)load_val(x, dtype, r0 + j) - (uint64_t)load_val(x, dtype, r0 + j - 1), wd);
                u[j] = ((uint64_t)d - (uint64_t)min_d) & msk;
                if (u[j] > umax) umax = u[j];
            }
            uint32_t b = orc_bits(umax);
            uint64_t len = align16(orc_packed_bytes(mk, b));
            if (pass == 1) {
                uint8_t* e = p + toff + 24ull * k;
                put_u64(e + 0, (uint64_t)base);
                put_u64(e + 8, (uint64_t)min_d);
                put_u32(e + 16, (uint32_t)poff);
                e[20] = (uint8_t)b; e[21] = e[22] = e[23] = 0;
                memset(p + sec1 + poff, 0, len);
                orc_pack(u, mk, b, p + sec1 + poff);
            }
            poff += len;
        }
        payload_total = poff;
    }
    free(u);
    return align16(w.end);
}

/* ---- RLE: maximal runs (value, count) + a row directory every 1024 rows ---- */
static uint64_t enc_rle(uint8_t* p, int dtype, const void* x, uint32_t m) {
    uint32_t R = 0;
    for (uint32_t i = 0; i < m; i++)
        if (i == 0 || load_val(x, dtype, i) != load_val(x, dtype, i - 1)) R++;
    uint32_t ntiles = (m + RLE_DIR_ROWS - 1) / RLE_DIR_ROWS;
    chunk_w w = {p, 64};
    chunk_header(p, ORC_RLE, dtype, 0, 0, m, R, 0);
    uint64_t voff = sec_begin(&w, 0, (uint64_t)R * size_of(dtype));
    uint64_t loff = sec_begin(&w, 1, (uint64_t)R * 4);
    uint64_t doff = sec_begin(&w, 2, (uint64_t)ntiles * 8);
    uint32_t r = 0, run_start = 0;
    for (uint32_t i = 0; i < m; i++) {
        if (i > 0 && load_val(x, dtype, i) != load_val(x, dtype, i - 1)) {
            put_u32(p + loff + 4ull * r, i - run_start);
            r++;
            run_start = i;
        }
        if (i == run_start) store_val(p + voff, dtype, r, (uint64_t)load_val(x, dtype, i));
        if (i % RLE_DIR_ROWS == 0) {
            put_u32(p + doff + 8ull * (i / RLE_DIR_ROWS), r);
            put_u32(p + doff + 8ull * (i / RLE_DIR_ROWS) + 4, i - run_start);
        }
    }
    if (m > 0) put_u32(p + loff + 4ull * r, m - run_start);
    return align16(w.end);
}

/* ---- LZ77: greedy, 4-byte hash of the last position, 64 KiB window ---- */
static uint32_t leb128_put(uint8_t* p, uint32_t v) {
    uint32_t n = 0;
    do { uint8_t c = v & 0x7F; v >>= 7; p[n++] = c | (v ? 0x80 : 0); } while (v);
    return n;
}
static uint32_t lz_hash(const uint8_t* s) {
    uint32_t v = (uint32_t)s[0] | ((uint32_t)s[1] << 8) | ((uint32_t)s[2] << 16) | ((uint32_t)s[3] << 24);
    return (v * 2654435761u) >> (32 - LZ_HASH_BITS);
}
static uint64_t enc_lz(uint8_t* p, const uint8_t* src, uint32_t m) {
    /* three streams: lengths (LEB128 literal length of every token and, between
     * them, match length - 4), u16 offsets, literal bytes */
    uint8_t* len = (uint8_t*)malloc(6ull * m + 16);
    uint8_t* offs = (uint8_t*)malloc(2ull * m + 16);
    uint8_t* lit = (uint8_t*)malloc((uint64_t)m + 16);
    int32_t* table = (int32_t*)malloc(sizeof(int32_t) << LZ_HASH_BITS);
    for (uint32_t i = 0; i < (1u << LZ_HASH_BITS); i++) table[i] = -1;
    uint32_t nl = 0, no = 0, ntok = 0, nlit = 0, lit_start = 0, pos = 0;
    while (pos + LZ_MIN_MATCH <= m) {
        uint32_t h = lz_hash(src + pos);
        int32_t cand = table[h];
        table[h] = (int32_t)pos;
        if (cand >= 0 && pos - (uint32_t)cand <= LZ_MAX_OFFSET &&
            memcmp(src + cand, src + pos, LZ_MIN_MATCH) == 0) {
            uint32_t mlen = LZ_MIN_MATCH;
            while (pos + mlen < m && src[cand + mlen] == src[pos + mlen]) mlen++;
            uint32_t ll = pos - lit_start;
            nl += leb128_put(len + nl, ll);
            memcpy(lit + nlit, src + lit_start, ll);
            nlit += ll;
            nl += leb128_put(len + nl, mlen - LZ_MIN_MATCH);
            put_u16(offs + no, pos - (uint32_t)cand);
            no += 2;
            ntok++;
            pos += mlen;
            lit_start = pos;
        } else {
            pos++;
        }
    }
    /* final token: the remaining literals, no match */
    uint32_t ll = m - lit_start;
    nl += leb128_put(len + nl, ll);
    memcpy(lit + nlit, src + lit_start, ll);
    nlit += ll;
    ntok++;
    chunk_w w = {p, 64};
    if ((uint64_t)nl + no + nlit >= m) {     /* does not compress: store the block raw */
        chunk_header(p, ORC_LZ77, ORC_BYTES, 0, 1, m, 0, 0);
        uint64_t off = sec_begin(&w, 0, m);
        memcpy(p + off, src, m);
    } else {
        chunk_header(p, ORC_LZ77, ORC_BYTES, 0, 0, m, ntok, 0);
        uint64_t a = sec_begin(&w, 0, nl);
        memcpy(p + a, len, nl);
        uint64_t b = sec_begin(&w, 1, no);
        if (no) memcpy(p + b, offs, no);
        uint64_t c = sec_begin(&w, 2, nlit);
        if (nlit) memcpy(p + c, lit, nlit);
    }
    free(len); free(offs); free(lit); free(table);
    return align16(w.end);
}

/* ---- Float2Int + bit-packing (Section 2.1 "Float2Int", Table 2) ----
 * A double v becomes the integer d with v = d / 10^e for a decimal exponent
 * e of the chunk (0..18); the integers are stored FOR + bit-packed.  The
 * decoded value of d is the double nearest to d / 10^e: for |d| <= 2^53 and
 * e <= 18 both d and 10^e are doubles exactly, so one IEEE division (which
 * rounds its exact quotient to nearest) is that value, written as the
 * definition says; a value that does not come back bit for bit from its rounded
 * integer (non-decimal values, NaN, infinities, -0.0, |v * 10^e| >= 2^53) is
 * an exception, stored as its row and its 64 bits.  The chunk's e has the
 * fewest exceptions (the smallest e on a tie). */
#define F2I_EMAX 18
#define F2I_DMAX 9007199254740992LL   /* 2^53 */
static double f2i_pow10(int e) {
    double p = 1.0;
    for (int k = 0; k < e; k++) p *= 10.0;   /* exact up to 10^22 */
    return p;
}
static double f2i_value(int64_t d, int e) {
    return (double)d / f2i_pow10(e);         /* exact operands: the correctly rounded quotient */
}
static int f2i_fits(double v, int e, int64_t* d) {
    if (!isfinite(v)) return 0;
    double t = v * f2i_pow10(e);
    if (!(fabs(t) < 9007199254740992.0)) return 0;
    int64_t k = (int64_t)nearbyint(t);        /* round half to even */
    double back = f2i_value(k, e);
    if (memcmp(&back, &v, 8) != 0) return 0;
    *d = k;
    return 1;
}
static uint64_t enc_f2i(uint8_t* p, const void* x, uint32_t m) {
    const double* v = (const double*)x;
    int best_e = 0;
    uint32_t best_ex = 0xFFFFFFFFu;
    for (int e = 0; e <= F2I_EMAX; e++) {
        uint32_t ex = 0;
        int64_t d;
        for (uint32_t i = 0; i < m; i++) ex += !f2i_fits(v[i], e, &d);
        if (ex < best_ex) { best_ex = ex; best_e = e; }
    }
    int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (m + 1));
    uint8_t* ok = (uint8_t*)malloc(m + 1);
    uint64_t* u = (uint64_t*)malloc(sizeof(uint64_t) * (m + 1));
    int64_t mn = 0;
    int have = 0;
    for (uint32_t i = 0; i < m; i++) {
        ok[i] = (uint8_t)f2i_fits(v[i], best_e, &d[i]);
        if (ok[i] && (!have || d[i] < mn)) { mn = d[i]; have = 1; }
    }
    uint64_t mx = 0;
    for (uint32_t i = 0; i < m; i++) {
        u[i] = ok[i] ? (uint64_t)d[i] - (uint64_t)mn : 0;
        if (u[i] > mx) mx = u[i];
    }
    uint32_t b = orc_bits(mx);
    chunk_w w = {p, 64};
    chunk_header(p, ORC_F2I, ORC_F64, b, 0, m, best_ex, (uint64_t)mn);
    p[48] = (uint8_t)best_e;
    uint64_t o0 = sec_begin(&w, 0, orc_packed_bytes(m, b));
    orc_pack(u, m, b, p + o0);
    uint64_t o1 = sec_begin(&w, 1, 4ull * best_ex);
    uint64_t o2 = sec_begin(&w, 2, 8ull * best_ex);
    uint32_t k = 0;
    for (uint32_t i = 0; i < m; i++)
        if (!ok[i]) {
            uint64_t bits;
            memcpy(&bits, &v[i], 8);
            put_u32(p + o1 + 4ull * k, i);
            put_u64(p + o2 + 8ull * k, bits);
            k++;
        }
    free(d);
    free(ok);
    free(u);
    return align16(w.end);
}


/* ---- dictionary + rANS ----
 * The chunk's distinct values (at most 256, sorted) are the symbols; each
 * row is coded as its rank.  rANS (Duda's range variant, byte-wise
 * renormalization): symbol s has frequency f_s >= 1 and cumulative frequency
 * c_s = f_0 + ... + f_{s-1} out of M; a state x maps to
 *   C(s, x) = floor(x / f_s) * M + (x mod f_s) + c_s
 * and back, with slot = x mod M and s the symbol whose [c_s, c_s + f_s)
 * holds the slot, to D(x) = f_s * floor(x / M) + slot - c_s.  States stay in
 * [L, 256 L): before C the encoder emits the low byte of x while
 * x >= (L / M) * 256 * f_s; after D the decoder reads a byte while x < L.
 * Every L rows form an independent stream (L = 2^k rows, k in 5..12, stored
 * in header byte 48; Section 5.2.3 varies the ANS chunk size to trade ratio
 * for throughput, and L is that size here): encoding runs from its last
 * row to its first starting at x = L; the stream is the final state (4 bytes,
 * little-endian) followed by the emitted bytes, last emitted first, so the
 * decoder reads it front to back and ends at x = L.
 * Sections: s0 = the sorted values; s1 = u16 f_s per symbol (padded to 4
 * bytes), then u32 start of each stream in s2 and the end of the last; s2 =
 * the streams.  Header: b = 12 (log2 M), n_aux = symbols, reference = streams. */

/* Frequencies out of M for counts cnt[0..nd) of n rows: f_s = max(1,
 * floor(cnt_s * M / n)); a shortfall goes to the most frequent symbol (the
 * first on a tie); an excess from the max(1) rule is taken one at a time
 * from the largest f_s above 1 (the first on a tie). */
static void ans_freqs(const uint32_t* cnt, uint32_t nd, uint32_t n, uint32_t* f) {
    uint64_t F = 0;
    for (uint32_t k = 0; k < nd; k++) {
        f[k] = (uint32_t)((uint64_t)cnt[k] * ANS_M / n);
        if (f[k] == 0) f[k] = 1;
        F += f[k];
    }
    if (F < ANS_M) {
        uint32_t best = 0;
        for (uint32_t k = 1; k < nd; k++)
            if (cnt[k] > cnt[best]) best = k;
        f[best] += (uint32_t)(ANS_M - F);
        F = ANS_M;
    }
    while (F > ANS_M) {
        uint32_t best = nd;
        for (uint32_t k = 0; k < nd; k++)
            if (f[k] > 1 && (best == nd || f[k] > f[best])) best = k;
        f[best]--;
        F--;
    }
}

/* one stream of n symbols; returns its length in bytes */
static uint32_t ans_encode(const uint32_t* sym, uint32_t n, const uint32_t* f, const uint32_t* c, uint8_t* out,
                           uint8_t* tmp) {
    uint32_t x = ANS_L, k = 0;
    for (uint32_t i = n; i-- > 0;) {
        uint32_t s = sym[i];
        uint64_t xmax = ((uint64_t)(ANS_L >> ANS_SCALE) << 8) * f[s];
        while (x >= xmax) { tmp[k++] = (uint8_t)(x & 0xFF); x >>= 8; }
        x = (x / f[s]) * ANS_M + (x % f[s]) + c[s];
    }
    put_u32(out, x);
    for (uint32_t j = 0; j < k; j++) out[4 + j] = tmp[k - 1 - j];
    return 4 + k;
}

static uint64_t enc_ans(uint8_t* p, int dtype, const void* x, uint32_t m, uint32_t L, int* err) {
    uint32_t lg = 0;
    while ((1u << lg) < L) lg++;
    if ((1u << lg) != L || lg < ANS_LOG_MIN || lg > ANS_LOG_MAX) { *err = ORC_EINVAL; return 0; }
    int64_t* s = (int64_t*)malloc(sizeof(int64_t) * (m ? m : 1));
    uint32_t* sym = (uint32_t*)malloc(sizeof(uint32_t) * (m ? m : 1));
    uint8_t* tmp = (uint8_t*)malloc(2ull * L + 16);
    uint8_t* streams = (uint8_t*)malloc(2ull * m + 8ull * (m / L + 1) + 16);
    if (!s || !sym || !tmp || !streams) { free(s); free(sym); free(tmp); free(streams); *err = ORC_ENOMEM; return 0; }
    for (uint32_t i = 0; i < m; i++) s[i] = load_val(x, dtype, i);
    qsort(s, m, sizeof(int64_t), cmp_i64);
    uint32_t nd = 0;
    for (uint32_t i = 0; i < m; i++)
        if (i == 0 || s[i] != s[nd - 1]) s[nd++] = s[i];
    if (nd > 256) { free(s); free(sym); free(tmp); free(streams); *err = ORC_EINVAL; return 0; }
    uint32_t cnt[256] = {0}, f[256], c[256];
    for (uint32_t i = 0; i < m; i++) {
        int64_t v = load_val(x, dtype, i);
        uint32_t lo = 0, hi = nd;
        while (lo < hi) { uint32_t mid = (lo + hi) / 2; if (s[mid] < v) lo = mid + 1; else hi = mid; }
        sym[i] = lo;
        cnt[lo]++;
    }
    if (nd) ans_freqs(cnt, nd, m, f);
    for (uint32_t k = 0, acc = 0; k < nd; k++) { c[k] = acc; acc += f[k]; }
    uint32_t K = (m + L - 1) / L;
    chunk_w w = {p, 64};
    chunk_header(p, ORC_ANS, dtype, ANS_SCALE, 0, m, nd, K);
    p[48] = (uint8_t)lg;
    uint64_t o0 = sec_begin(&w, 0, (uint64_t)nd * size_of(dtype));
    for (uint32_t k = 0; k < nd; k++) store_val(p + o0, dtype, k, (uint64_t)s[k]);
    uint64_t fbytes = (2ull * nd + 3) / 4 * 4;
    uint64_t o1 = sec_begin(&w, 1, fbytes + 4ull * (K + 1));
    for (uint32_t k = 0; k < nd; k++) put_u16(p + o1 + 2ull * k, f[k]);
    uint64_t pos = 0;
    for (uint32_t j = 0; j < K; j++) {
        uint32_t r0 = j * L, n = m - r0 < L ? m - r0 : L;
        put_u32(p + o1 + fbytes + 4ull * j, (uint32_t)pos);
        pos += ans_encode(sym + r0, n, f, c, streams + pos, tmp);
    }
    put_u32(p + o1 + fbytes + 4ull * K, (uint32_t)pos);
    uint64_t o2 = sec_begin(&w, 2, pos);
    memcpy(p + o2, streams, pos);
    free(s); free(sym); free(tmp); free(streams);
    return align16(w.end);
}

/* ---- string dictionary + bit-packing (bytes) ----
 * The chunk's bytes are cut into tokens: a token ends after a space byte,
 * before the first byte of a row, after STR_TOKEN_MAX bytes, or at the end of
 * the chunk.  The dictionary is the distinct tokens in byte order (a prefix
 * first); each token is stored as its rank, bit-packed at bits(ndict - 1).
 * With more than STR_DICT_MAX distinct tokens every byte is a token instead.
 * Sections: s0 = dictionary offsets [ndict + 1] then the output offset of
 * every STR_TILE-th token; s1 = the dictionary's bytes; s2 = the codes. */
typedef struct { const uint8_t* s; uint32_t len; } str_tok;

static int cmp_tok(const void* a, const void* b) {
    const str_tok* x = (const str_tok*)a;
    const str_tok* y = (const str_tok*)b;
    uint32_t n = x->len < y->len ? x->len : y->len;
    int c = n ? memcmp(x->s, y->s, n) : 0;
    if (c) return c;
    return (x->len > y->len) - (x->len < y->len);
}

static uint32_t str_tokens(const uint8_t* x, uint32_t m, const uint8_t* row_start, int bytes_only, str_tok* t) {
    uint32_t n = 0, i = 0;
    while (i < m) {
        uint32_t j = i + 1;
        if (!bytes_only)
            while (j < m && x[j - 1] != ' ' && !row_start[j] && j - i < STR_TOKEN_MAX) j++;
        t[n].s = x + i;
        t[n].len = j - i;
        n++;
        i = j;
    }
    return n;
}

/* sorted distinct tokens of t[0..n) into d; returns their number */
static uint32_t str_dict(const str_tok* t, uint32_t n, str_tok* d) {
    memcpy(d, t, sizeof(str_tok) * n);
    qsort(d, n, sizeof(str_tok), cmp_tok);
    uint32_t nd = 0;
    for (uint32_t i = 0; i < n; i++)
        if (nd == 0 || cmp_tok(&d[nd - 1], &d[i]) != 0) d[nd++] = d[i];
    return nd;
}

static uint64_t enc_strdict(uint8_t* p, const uint8_t* x, uint32_t m, const uint8_t* row_start, int* err) {
    str_tok* t = (str_tok*)malloc(sizeof(str_tok) * (m ? m : 1));
    str_tok* d = (str_tok*)malloc(sizeof(str_tok) * (m ? m : 1));
    if (!t || !d) { free(t); free(d); *err = ORC_ENOMEM; return 0; }
    uint32_t T = str_tokens(x, m, row_start, 0, t);
    uint32_t nd = str_dict(t, T, d);
    if (nd > STR_DICT_MAX) {
        T = str_tokens(x, m, row_start, 1, t);
        nd = str_dict(t, T, d);
    }
    uint32_t b = orc_bits(nd ? nd - 1 : 0), ntiles = (T + STR_TILE - 1) / STR_TILE;
    uint64_t dbytes = 0;
    for (uint32_t k = 0; k < nd; k++) dbytes += d[k].len;
    chunk_w w = {p, 64};
    chunk_header(p, ORC_STRDICT, ORC_BYTES, b, 0, m, nd, T);
    uint64_t o0 = sec_begin(&w, 0, 4ull * (nd + 1 + ntiles));
    uint64_t o1 = sec_begin(&w, 1, dbytes);
    uint64_t pos = 0;
    for (uint32_t k = 0; k < nd; k++) {
        put_u32(p + o0 + 4ull * k, (uint32_t)pos);
        memcpy(p + o1 + pos, d[k].s, d[k].len);
        pos += d[k].len;
    }
    put_u32(p + o0 + 4ull * nd, (uint32_t)pos);
    uint64_t* code = (uint64_t*)malloc(sizeof(uint64_t) * (T ? T : 1));
    if (!code) { free(t); free(d); *err = ORC_ENOMEM; return 0; }
    uint64_t out_pos = 0;
    for (uint32_t i = 0; i < T; i++) {
        const str_tok* hit = (const str_tok*)bsearch(&t[i], d, nd, sizeof(str_tok), cmp_tok);
        code[i] = (uint64_t)(hit - d);
        if (i % STR_TILE == 0) put_u32(p + o0 + 4ull * (nd + 1 + i / STR_TILE), (uint32_t)out_pos);
        out_pos += t[i].len;
    }
    uint64_t o2 = sec_begin(&w, 2, orc_packed_bytes(T, b));
    orc_pack(code, T, b, p + o2);
    free(code);
    free(t);
    free(d);
    return align16(w.end);
}

/* ------------------------------------------------------------------------- */
/* column encoder                                                            */
/* ------------------------------------------------------------------------- */
uint64_t orc_encode_bound(int scheme, int dtype, uint64_t n, uint32_t chunk_rows) {
    if (chunk_rows == 0) return 0;
    uint64_t nch = (n + chunk_rows - 1) / chunk_rows;
    return 64 + 32 * nch + nch * chunk_bound(scheme, dtype, chunk_rows) + 64;
}

static int scheme_ok(int scheme, int dtype) {
    if (dtype == ORC_BYTES) return scheme == ORC_RAW || scheme == ORC_LZ77 || scheme == ORC_STRDICT;
    if (dtype == ORC_F64) return scheme == ORC_RAW || scheme == ORC_F2I;
    if (dtype != ORC_I32 && dtype != ORC_I64) return 0;
    return (scheme >= ORC_RAW && scheme <= ORC_RLE) || scheme == ORC_ANS;
}

/* Column assembly shared by orc_encode and orc_encode_ans. */
static int encode_column(int scheme, int dtype, const void* data, uint64_t n, uint32_t chunk_rows,
                         uint32_t ans_stream, uint8_t* out, uint64_t cap, uint64_t* out_len) {
    if (!scheme_ok(scheme, dtype) || chunk_rows == 0) return ORC_EINVAL;
    if (cap < orc_encode_bound(scheme, dtype, n, chunk_rows)) return ORC_EINVAL;
    uint64_t nch = (n + chunk_rows - 1) / chunk_rows;
    uint64_t sz = size_of(dtype);
    memset(out, 0, cap);               /* every padding byte is zero */
    uint64_t pos = 64 + 32 * nch;
    for (uint64_t c = 0; c < nch; c++) {
        uint64_t r0 = c * chunk_rows;
        uint32_t m = (uint32_t)(n - r0 < chunk_rows ? n - r0 : chunk_rows);
        const uint8_t* x = (const uint8_t*)data + r0 * sz;
        uint8_t* p = out + pos;
        int err = ORC_OK;
        uint64_t len = 0;
        switch (scheme) {
        case ORC_RAW: len = enc_raw(p, dtype, x, m); break;
        case ORC_FOR_BP: len = enc_for(p, dtype, x, m); break;
        case ORC_DICT_BP: len = enc_dict(p, dtype, x, m, &err); break;
        case ORC_DELTA_BP: len = enc_delta(p, dtype, x, m); break;
        case ORC_RLE: len = enc_rle(p, dtype, x, m); break;
        case ORC_LZ77: len = enc_lz(p, x, m); break;
        case ORC_F2I: len = enc_f2i(p, x, m); break;
        case ORC_STRDICT: return ORC_EINVAL;   /* needs the row offsets: orc_encode_strdict */
        case ORC_ANS: len = enc_ans(p, dtype, x, m, ans_stream, &err); break;
        }
        if (err) return err;
        uint8_t* d = out + 64 + 32 * c;
        put_u64(d + 0, pos);
        put_u64(d + 8, len);
        put_u64(d + 16, r0);
        put_u32(d + 24, m);
        put_u32(d + 28, 0);
        pos += len;
    }
    put_u32(out + 0, COL_MAGIC);
    put_u16(out + 4, 1);
    out[6] = (uint8_t)scheme;
    out[7] = (uint8_t)dtype;
    put_u32(out + 8, (uint32_t)nch);
    put_u32(out + 12, chunk_rows);
    put_u64(out + 16, n);
    put_u64(out + 24, n * sz);
    put_u64(out + 32, pos);
    *out_len = pos;
    return ORC_OK;
}

/* Encode n values (BYTES: n bytes) in chunks of chunk_rows rows (ANS:
 * streams of 512 rows).  `out` must hold orc_encode_bound(...) bytes.
 * *out_len receives the size. */
int orc_encode(int scheme, int dtype, const void* data, uint64_t n, uint32_t chunk_rows,
               uint8_t* out, uint64_t cap, uint64_t* out_len) {
    return encode_column(scheme, dtype, data, n, chunk_rows, ANS_SUB_DEFAULT, out, cap, out_len);
}

/* The same for dictionary + ANS with `stream_rows` rows per independent
 * stream (a power of two, 32 .. 4096). */
int orc_encode_ans(int dtype, const void* data, uint64_t n, uint32_t chunk_rows, uint32_t stream_rows,
                   uint8_t* out, uint64_t cap, uint64_t* out_len) {
    return encode_column(ORC_ANS, dtype, data, n, chunk_rows, stream_rows, out, cap, out_len);
}


/* A byte column of n bytes whose rows start at offsets[0..nrows] (offsets[0]
 * = 0, offsets[nrows] = n, nondecreasing) in string-dictionary chunks of
 * chunk_bytes bytes.  `out` must hold orc_encode_bound(ORC_STRDICT,
 * ORC_BYTES, n, chunk_bytes) bytes. */
int orc_encode_strdict(const uint8_t* data, uint64_t n, const int32_t* offsets, uint64_t nrows,
                       uint32_t chunk_bytes, uint8_t* out, uint64_t cap, uint64_t* out_len) {
    if (chunk_bytes == 0 || cap < orc_encode_bound(ORC_STRDICT, ORC_BYTES, n, chunk_bytes)) return ORC_EINVAL;
    if (offsets[0] != 0 || (uint64_t)offsets[nrows] != n) return ORC_EINVAL;
    for (uint64_t r = 0; r < nrows; r++)
        if (offsets[r + 1] < offsets[r]) return ORC_EINVAL;
    uint64_t nch = (n + chunk_bytes - 1) / chunk_bytes;
    memset(out, 0, cap);
    uint8_t* row_start = (uint8_t*)malloc(chunk_bytes + 1);
    if (!row_start) return ORC_ENOMEM;
    uint64_t pos = 64 + 32 * nch, r = 0;
    for (uint64_t c = 0; c < nch; c++) {
        uint64_t c0 = c * chunk_bytes;
        uint32_t m = (uint32_t)(n - c0 < chunk_bytes ? n - c0 : chunk_bytes);
        memset(row_start, 0, (size_t)m + 1);
        while (r <= nrows && (uint64_t)offsets[r] < c0) r++;
        for (uint64_t q = r; q <= nrows && (uint64_t)offsets[q] < c0 + m; q++) row_start[offsets[q] - c0] = 1;
        int err = ORC_OK;
        uint64_t len = enc_strdict(out + pos, data + c0, m, row_start, &err);
        if (err) { free(row_start); return err; }
        uint8_t* d = out + 64 + 32 * c;
        put_u64(d + 0, pos);
        put_u64(d + 8, len);
        put_u64(d + 16, c0);
        put_u32(d + 24, m);
        put_u32(d + 28, 0);
        pos += len;
    }
    free(row_start);
    put_u32(out + 0, COL_MAGIC);
    put_u16(out + 4, 1);
    out[6] = (uint8_t)ORC_STRDICT;
    out[7] = (uint8_t)ORC_BYTES;
    put_u32(out + 8, (uint32_t)nch);
    put_u32(out + 12, chunk_bytes);
    put_u64(out + 16, n);
    put_u64(out + 24, n);
    put_u64(out + 32, pos);
    *out_len = pos;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* decoders                                                                  */
/* ------------------------------------------------------------------------- */
/* a section lies inside the blob */
static int sec_ok(const uint8_t* c, uint64_t len, int s) {
    uint64_t off = get_u32(c + 24 + 4 * s), l = get_u32(c + 36 + 4 * s);
    return off >= 64 && off % 16 == 0 && off + l <= len;
}

/* Decode one chunk blob into `out` (rows values).  Returns ORC_ECORRUPT for a
 * malformed blob. */
int orc_decode_chunk(const uint8_t* c, uint64_t len, void* out, uint64_t out_cap) {
    if (len < 64 || get_u32(c) != CHK_MAGIC) return ORC_ECORRUPT;
    int scheme = c[4], dtype = c[5];
    uint32_t b = c[6], flags = c[7], m = get_u32(c + 8), n_aux = get_u32(c + 12);
    uint64_t ref = get_u64(c + 16);
    if (!scheme_ok(scheme, dtype)) return ORC_ECORRUPT;
    unsigned wd = width_of(dtype);
    uint64_t msk = mask_of(wd), sz = size_of(dtype);
    if ((uint64_t)m * sz > out_cap) return ORC_EINVAL;
    const uint8_t* s0 = c + get_u32(c + 24);
    const uint8_t* s1 = c + get_u32(c + 28);
    const uint8_t* s2 = c + get_u32(c + 32);
    uint32_t l0 = get_u32(c + 36), l1 = get_u32(c + 40), l2 = get_u32(c + 44);
    switch (scheme) {
    case ORC_RAW:
        if (!sec_ok(c, len, 0) || l0 != (uint64_t)m * sz) return ORC_ECORRUPT;
        memcpy(out, s0, (uint64_t)m * sz);
        return ORC_OK;
    case ORC_FOR_BP:
        /* x_i = reference + unpacked value i */
        if (!sec_ok(c, len, 0) || b > wd || l0 != orc_packed_bytes(m, b)) return ORC_ECORRUPT;
        for (uint32_t i = 0; i < m; i++) store_val(out, dtype, i, (ref + orc_unpack_one(s0, i, b)) & msk);
        return ORC_OK;
    case ORC_DICT_BP:
        /* x_i = dictionary[code_i] */
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || b > 16 || l0 != (uint64_t)n_aux * sz ||
            l1 != orc_packed_bytes(m, b)) return ORC_ECORRUPT;
        for (uint32_t i = 0; i < m; i++) {
            uint64_t code = orc_unpack_one(s1, i, b);
            if (code >= n_aux) return ORC_ECORRUPT;
            store_val(out, dtype, i, (uint64_t)load_val(s0, dtype, code));
        }
        return ORC_OK;
    case ORC_DELTA_BP: {
        /* x_0 = base; x_j = x_{j-1} + (min_d + u_j) */
        uint32_t nb = n_aux;
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || nb != (m + DELTA_BLOCK - 1) / DELTA_BLOCK ||
            l0 != 24ull * nb) return ORC_ECORRUPT;
        for (uint32_t k = 0; k < nb; k++) {
            const uint8_t* e = s0 + 24ull * k;
            uint64_t base = get_u64(e), min_d = get_u64(e + 8);
            uint32_t poff = get_u32(e + 16), bk = e[20];
            uint32_t r0 = k * DELTA_BLOCK;
            uint32_t mk = m - r0 < DELTA_BLOCK ? m - r0 : DELTA_BLOCK;
            if (bk > wd || (uint64_t)poff + orc_packed_bytes(mk, bk) > l1) return ORC_ECORRUPT;
            uint64_t prev = base & msk;
            store_val(out, dtype, r0, prev);
            for (uint32_t j = 1; j < mk; j++) {
                prev = (prev + min_d + orc_unpack_one(s1 + poff, j, bk)) & msk;
                store_val(out, dtype, r0 + j, prev);
            }
        }
        return ORC_OK;
    }
    case ORC_RLE: {
        /* presum = exclusive prefix sum of counts; run r fills [presum_r, presum_r + count_r) */
        uint32_t R = n_aux;
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || !sec_ok(c, len, 2) ||
            l0 != (uint64_t)R * sz || l1 != 4ull * R) return ORC_ECORRUPT;
        uint64_t presum = 0;
        for (uint32_t r = 0; r < R; r++) {
            uint32_t cnt = get_u32(s1 + 4ull * r);
            if (cnt == 0 || presum + cnt > m) return ORC_ECORRUPT;
            uint64_t v = (uint64_t)load_val(s0, dtype, r);
            for (uint32_t k = 0; k < cnt; k++) store_val(out, dtype, presum + k, v);
            presum += cnt;
        }
        if (presum != m) return ORC_ECORRUPT;
        (void)s2; (void)l2;
        return ORC_OK;
    }
    case ORC_F2I: {
        /* v_i = f2i_value(ref + u_i, e); the rows listed in s1 take the 64 bits in s2.
         * The encoder's integers satisfy |d| <= 2^53 (|v * 10^e| < 2^53, rounded):
         * a stream with a larger one is malformed. */
        uint32_t e = c[48];
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || !sec_ok(c, len, 2) || b > 64 || e > F2I_EMAX ||
            n_aux > m || l0 != orc_packed_bytes(m, b) || l1 != 4ull * n_aux || l2 != 8ull * n_aux)
            return ORC_ECORRUPT;
        double* o = (double*)out;
        for (uint32_t i = 0; i < m; i++) {
            int64_t d = (int64_t)(ref + orc_unpack_one(s0, i, b));
            if (d > F2I_DMAX || d < -F2I_DMAX) return ORC_ECORRUPT;
            o[i] = f2i_value(d, (int)e);
        }
        for (uint32_t k = 0; k < n_aux; k++) {
            uint32_t pos = get_u32(s1 + 4ull * k);
            if (pos >= m || (k > 0 && pos <= get_u32(s1 + 4ull * (k - 1)))) return ORC_ECORRUPT;
            uint64_t bits = get_u64(s2 + 8ull * k);
            memcpy(&o[pos], &bits, 8);
        }
        return ORC_OK;
    }
    case ORC_ANS: {
        /* each stream: read the state, then per row find the symbol of slot
         * x mod M, emit its value, step x = f * (x / M) + slot - c and read
         * bytes while x < L; the stream must end at x = L with every byte read */
        uint32_t nd = n_aux;
        uint64_t K = ref, fbytes = (2ull * nd + 3) / 4 * 4;
        uint32_t lg = c[48];
        if (lg < ANS_LOG_MIN || lg > ANS_LOG_MAX) return ORC_ECORRUPT;
        uint32_t L = 1u << lg;
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || !sec_ok(c, len, 2) || b != ANS_SCALE || nd == 0 ||
            nd > 256 || l0 != (uint64_t)nd * sz || K != (m + L - 1) / L || l1 != fbytes + 4 * (K + 1))
            return ORC_ECORRUPT;
        uint32_t f[256], cum[256], acc = 0;
        for (uint32_t k = 0; k < nd; k++) {
            f[k] = get_u16(s1 + 2ull * k);
            if (f[k] == 0) return ORC_ECORRUPT;
            cum[k] = acc;
            acc += f[k];
        }
        if (acc != ANS_M) return ORC_ECORRUPT;
        const uint8_t* st = s1 + fbytes;
        if (get_u32(st) != 0 || get_u32(st + 4 * K) != l2) return ORC_ECORRUPT;
        for (uint64_t j = 0; j < K; j++) {
            uint32_t a0 = get_u32(st + 4 * j), a1 = get_u32(st + 4 * (j + 1));
            if (a1 < a0 || a1 - a0 < 4) return ORC_ECORRUPT;
            const uint8_t* q = s2 + a0;
            uint32_t ql = a1 - a0, qp = 4, x = get_u32(q);
            uint32_t r0 = (uint32_t)j * L, n = m - r0 < L ? m - r0 : L;
            for (uint32_t i = 0; i < n; i++) {
                uint32_t slot = x & (ANS_M - 1), sym = 0;
                while (!(cum[sym] <= slot && slot < cum[sym] + f[sym])) sym++;
                store_val(out, dtype, r0 + i, (uint64_t)load_val(s0, dtype, sym) & msk);
                x = f[sym] * (x >> ANS_SCALE) + slot - cum[sym];
                while (x < ANS_L) {
                    if (qp >= ql) return ORC_ECORRUPT;
                    x = (x << 8) | q[qp++];
                }
            }
            if (x != ANS_L || qp != ql) return ORC_ECORRUPT;
        }
        (void)flags;
        return ORC_OK;
    }
    case ORC_STRDICT: {
        /* the output is the dictionary entries of the codes, one after another */
        uint8_t* o = (uint8_t*)out;
        uint32_t nd = n_aux;
        uint64_t T = ref, ntiles = (T + STR_TILE - 1) / STR_TILE;
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || !sec_ok(c, len, 2) || nd == 0 || nd > STR_DICT_MAX ||
            b != orc_bits(nd - 1) || T > m || (m > 0 && T == 0) || l0 != 4ull * (nd + 1 + ntiles) ||
            l2 != orc_packed_bytes(T, b))
            return ORC_ECORRUPT;
        if (get_u32(s0) != 0 || get_u32(s0 + 4ull * nd) != l1) return ORC_ECORRUPT;
        for (uint32_t k = 0; k < nd; k++) {
            uint32_t a0 = get_u32(s0 + 4ull * k), a1 = get_u32(s0 + 4ull * (k + 1));
            if (a1 <= a0 || a1 - a0 > STR_TOKEN_MAX) return ORC_ECORRUPT;
        }
        uint64_t op = 0;
        for (uint64_t t = 0; t < T; t++) {
            if (t % STR_TILE == 0 && get_u32(s0 + 4ull * (nd + 1 + t / STR_TILE)) != op) return ORC_ECORRUPT;
            uint64_t k = orc_unpack_one(s2, t, b);
            if (k >= nd) return ORC_ECORRUPT;
            uint32_t a0 = get_u32(s0 + 4 * k), a1 = get_u32(s0 + 4 * (k + 1));
            if (op + (a1 - a0) > m) return ORC_ECORRUPT;
            for (uint32_t q = a0; q < a1; q++) o[op++] = s1[q];
        }
        if (op != m) return ORC_ECORRUPT;
        (void)flags;
        return ORC_OK;
    }
    case ORC_LZ77: {
        uint8_t* o = (uint8_t*)out;
        if (flags & 1) {
            if (!sec_ok(c, len, 0) || l0 != m) return ORC_ECORRUPT;
            memcpy(o, s0, m);
            return ORC_OK;
        }
        /* token t: literal length (varint 2t), the literals, then unless t is the
         * last token a back-reference: offset t, length varint 2t+1 plus 4 */
        if (!sec_ok(c, len, 0) || !sec_ok(c, len, 1) || !sec_ok(c, len, 2) || n_aux == 0 ||
            l1 != 2ull * (n_aux - 1)) return ORC_ECORRUPT;
        uint32_t vp = 0, lp = 0, op = 0;
        for (uint32_t t = 0; t < n_aux; t++) {
            uint32_t ll = 0, sh = 0;
            for (;;) {
                if (vp >= l0 || sh > 14) return ORC_ECORRUPT; /* at most 3 bytes */
                uint8_t byte = s0[vp++];
                ll |= (uint32_t)(byte & 0x7F) << sh;
                sh += 7;
                if (!(byte & 0x80)) break;
            }
            if ((uint64_t)lp + ll > l2 || (uint64_t)op + ll > m) return ORC_ECORRUPT;
            for (uint32_t k = 0; k < ll; k++) o[op++] = s2[lp++];
            if (t + 1 == n_aux) break;
            uint32_t ml = 0;
            sh = 0;
            for (;;) {
                if (vp >= l0 || sh > 14) return ORC_ECORRUPT; /* at most 3 bytes */
                uint8_t byte = s0[vp++];
                ml |= (uint32_t)(byte & 0x7F) << sh;
                sh += 7;
                if (!(byte & 0x80)) break;
            }
            ml += LZ_MIN_MATCH;
            uint32_t off = get_u16(s1 + 2ull * t);
            if (off == 0 || off > op || (uint64_t)op + ml > m) return ORC_ECORRUPT;
            /* back-reference: byte by byte, so a source that overlaps the output repeats */
            for (uint32_t k = 0; k < ml; k++) { o[op] = o[op - off]; op++; }
        }
        if (op != m || vp != l0 || lp != l2) return ORC_ECORRUPT;
        return ORC_OK;
    }
    }
    return ORC_ECORRUPT;
}

/* header fields of a serialized column */
int orc_column_info(const uint8_t* buf, uint64_t len, uint32_t* scheme, uint32_t* dtype,
                    uint64_t* n_rows, uint32_t* n_chunks, uint64_t* total) {
    if (len < 64 || get_u32(buf) != COL_MAGIC || get_u16(buf + 4) != 1) return ORC_ECORRUPT;
    *scheme = buf[6];
    *dtype = buf[7];
    *n_chunks = get_u32(buf + 8);
    *n_rows = get_u64(buf + 16);
    *total = get_u64(buf + 32);
    return ORC_OK;
}

/* Decode a serialized column into `out`. */
int orc_decode(const uint8_t* buf, uint64_t len, void* out, uint64_t out_cap) {
    uint32_t scheme, dtype, nch;
    uint64_t n, total;
    int st = orc_column_info(buf, len, &scheme, &dtype, &n, &nch, &total);
    if (st) return st;
    uint64_t sz = size_of((int)dtype);
    if (total > len || 64 + 32ull * nch > total) return ORC_ECORRUPT;
    if (n * sz > out_cap) return ORC_EINVAL;
    uint64_t rows_seen = 0;
    for (uint32_t c = 0; c < nch; c++) {
        const uint8_t* d = buf + 64 + 32ull * c;
        uint64_t off = get_u64(d), l = get_u64(d + 8), r0 = get_u64(d + 16);
        uint32_t m = get_u32(d + 24);
        if (off + l > total || r0 != rows_seen || r0 + m > n) return ORC_ECORRUPT;
        if (get_u32(buf + off + 8) != m) return ORC_ECORRUPT;
        st = orc_decode_chunk(buf + off, l, (uint8_t*)out + r0 * sz, (n - r0) * sz);
        if (st) return st;
        rows_seen += m;
    }
    return rows_seen == n ? ORC_OK : ORC_ECORRUPT;
}

/* Byte offset and length of chunk c of a serialized column. */
int orc_chunk_span(const uint8_t* buf, uint64_t len, uint32_t c, uint64_t* off, uint64_t* l,
                   uint64_t* row0, uint32_t* rows) {
    if (len < 64 || get_u32(buf) != COL_MAGIC || c >= get_u32(buf + 8)) return ORC_EINVAL;
    const uint8_t* d = buf + 64 + 32ull * c;
    *off = get_u64(d);
    *l = get_u64(d + 8);
    *row0 = get_u64(d + 16);
    *rows = get_u32(d + 24);
    return ORC_OK;
}
