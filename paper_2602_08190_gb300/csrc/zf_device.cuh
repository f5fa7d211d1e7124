// zf_device.cuh -- device-side decode of one warp job: up to K consecutive
// 1024-row warp tiles of one chunk, per scheme.
//
// A launch decodes a list of chunks (ZfDevChunk) cut into warp jobs.  Each
// warp decodes its job alone, in its own slice of shared memory, with no
// CTA-wide barrier.  Inside a job the warp fetches all block / directory
// metadata of its tiles at once and copies the next tile's compressed bytes
// into shared memory (cp.async, double-buffered) while it decodes the
// current tile, so DRAM latency overlaps the decode.  The decoders follow
// the parallel patterns of Section 3.1:
//   fp_job      Fully-Parallel: FOR / dictionary / Float2Int / raw.  Every
//               lane extracts C = 16/sizeof(T) consecutive values of the
//               staged bits with funnel shifts and writes them with one
//               16-byte store (coalesced).  Float2Int makes each integer
//               the double nearest d / 10^e with integer multiplies
//               (zf_f2i.h) and then patches the chunk's exceptions.
//   delta_job   Group-Parallel: one 1024-row block per step.  Lane l owns
//               values [32l, 32l+32): it sums its differences, one warp
//               shuffle scan gives every lane its offset, the values are
//               rebuilt from a second read of the differences and leave
//               through a shared-memory transpose, four lanes per 128-byte line.
//   rle_job     Group-Parallel: the tile's run lengths (the chunk's 1024-row
//               directory names the first run) are scanned into start rows,
//               four per lane and one warp shuffle scan per 128 runs (the
//               presum of Section 3.2); every run but the first sets its start
//               row's bit in a 32-word bitmask, and a row's run is the number
//               of set bits at or before it.  Each tile writes exactly 1024
//               rows, so long and short runs balance.
//   strdict_job (zf_strdict.cuh) Group-Parallel: string-dictionary tokens
//               of a byte column, placed by one warp scan of their lengths.
// A failed check of the stream sets a bit in the launch's error word; the
// tile then writes in-bounds placeholder values.  Nothing traps.
#pragma once
#include <cuda_pipeline.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "zf_f2i.h"
#include "zf_internal.h"

namespace zfd {

// Reciprocals of 5^e for the Float2Int value (zf_f2i.h); a warp job reads one
// row, the same for all its lanes.
static __constant__ zf::F2IRecip kF2IRecip[zf::kF2IMaxExp + 1] = {ZF_F2I_RECIP_ROWS};

constexpr uint32_t kWarpRows = 1024;

struct Hdr {
    uint32_t rows, n_aux, b, flags;
    uint64_t ref;
    uint32_t off[3], len[3];
};

__device__ __forceinline__ uint4 ldg16(const void* p) { return __ldg(reinterpret_cast<const uint4*>(p)); }

__device__ __forceinline__ void load_hdr(const uint8_t* blob, Hdr& h) {
    uint4 a = ldg16(blob), b = ldg16(blob + 16), c = ldg16(blob + 32);
    h.b = (a.y >> 16) & 0xFF;
    h.flags = a.y >> 24;
    h.rows = a.z;
    h.n_aux = a.w;
    h.ref = ((uint64_t)b.y << 32) | b.x;
    h.off[0] = b.z;
    h.off[1] = b.w;
    h.off[2] = c.x;
    h.len[0] = c.y;
    h.len[1] = c.z;
    h.len[2] = c.w;
}

__device__ __forceinline__ void report(uint32_t* err, uint32_t code, uint32_t chunk_id) {
    atomicOr(&err[0], 1u << code);
    atomicCAS(&err[1], 0xFFFFFFFFu, chunk_id);
}

// Bits [bitpos, bitpos + b) of a little-endian word stream in shared memory.
__device__ __forceinline__ uint64_t extract(const uint32_t* sm, uint32_t bitpos, uint32_t b) {
    uint32_t w = bitpos >> 5, sh = bitpos & 31;
    uint32_t w0 = sm[w], w1 = sm[w + 1];
    uint32_t lo = __funnelshift_r(w0, w1, sh);
    if (b <= 32) return b == 32 ? lo : (lo & ((1u << b) - 1u));
    uint32_t hi = __funnelshift_r(w1, sm[w + 2], sh);
    uint64_t v = ((uint64_t)hi << 32) | lo;
    return b == 64 ? v : (v & ((1ull << b) - 1ull));
}

// One 256-bit store of four 64-bit words to a 32-byte aligned global address:
// a lane writes a whole L2 sector at once.  st.global takes a global-space
// address, so the generic pointer is converted first.  The decoders that use
// it are inlined into their kernels (the batched kernel included): inside a
// function called out of line (through the ABI) the same store was seen to
// write only its first word on sm_103a, so no out-of-line function uses it
// (WS = false there, as in delta_block_wide and the allocation-free kernel).
__device__ __forceinline__ void store32(void* dst, unsigned long long a, unsigned long long b, unsigned long long c,
                                        unsigned long long d) {
    const size_t g = __cvta_generic_to_global(dst);
    asm volatile("st.global.v4.b64 [%0], {%1, %2, %3, %4};" ::"l"(g), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

// Store N consecutive values of type T with the widest aligned vector stores
// (the values are packed into 32-bit words in registers first).  32-byte rows
// use one 256-bit store when `al32` says the address is 32-byte aligned, so
// a lane writes a whole L2 sector at once.
template <class T, int N>
__device__ __forceinline__ void store_vec(T* dst, const T (&v)[N], bool al32 = false) {
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "int32 or int64 values");
    constexpr int W = N * (int)sizeof(T) / 4;
    uint32_t w[W];
#pragma unroll
    for (int k = 0; k < N; k++) {
        if constexpr (sizeof(T) == 8) {
            w[2 * k] = (uint32_t)(uint64_t)v[k];
            w[2 * k + 1] = (uint32_t)((uint64_t)v[k] >> 32);
        } else {
            w[k] = (uint32_t)v[k];
        }
    }
    if constexpr (W == 8) {
        if (al32) {
            store32(dst, ((unsigned long long)w[1] << 32) | w[0], ((unsigned long long)w[3] << 32) | w[2],
                    ((unsigned long long)w[5] << 32) | w[4], ((unsigned long long)w[7] << 32) | w[6]);
            return;
        }
    }
    if constexpr (W % 4 == 0) {
#pragma unroll
        for (int q = 0; q < W / 4; q++)
            reinterpret_cast<uint4*>(dst)[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
    } else if constexpr (W % 2 == 0) {
#pragma unroll
        for (int q = 0; q < W / 2; q++) reinterpret_cast<uint2*>(dst)[q] = make_uint2(w[2 * q], w[2 * q + 1]);
    } else {
#pragma unroll
        for (int q = 0; q < W; q++) reinterpret_cast<uint32_t*>(dst)[q] = w[q];
    }
}

template <class S>
__device__ __forceinline__ S warp_incl_sum(S x, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        S y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    return x;
}

// Inclusive sum over the lanes of values <= cap, saturating at cap (cap <
// 2^31, so no partial sum wraps).
__device__ __forceinline__ uint32_t warp_incl_sum_sat(uint32_t x, uint32_t cap, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x = min(x + y, cap);
    }
    return x;
}

// ---------------------------------------------------------------- async staging
// Copy `nbytes` (rounded up to 16) from a 16-byte aligned global address into
// a warp's shared-memory buffer with cp.async, 16 bytes per lane per step.
// The caller commits the group.
__device__ __forceinline__ void stage_async(uint32_t* buf, const uint8_t* src, uint32_t nbytes, uint32_t lane) {
    const uint32_t nvec = (nbytes + 15) >> 4;
    for (uint32_t i = lane; i < nvec; i += 32) __pipeline_memcpy_async(buf + 4 * i, src + 16ull * i, 16);
}

// Four consecutive b-bit values starting at bit `bitpos`.  NARROW needs
// b <= 8 (4b + 31 <= 63: one 64-bit window of two words).
template <bool NARROW, class S>
__device__ __forceinline__ void extract4(const uint32_t* wsm, uint32_t bitpos, uint32_t b, S (&u)[4]) {
    if constexpr (NARROW) {
        const uint32_t w = bitpos >> 5, sh = bitpos & 31;
        const uint64_t x = ((((uint64_t)wsm[w + 1]) << 32) | wsm[w]) >> sh;
        const uint32_t m = (1u << b) - 1u;
#pragma unroll
        for (int k = 0; k < 4; k++) u[k] = (S)((uint32_t)(x >> (k * b)) & m);
    } else {
#pragma unroll
        for (int k = 0; k < 4; k++) u[k] = (S)extract(wsm, bitpos + k * b, b);
    }
}

// Bytes of one staging buffer of a warp for packed payloads of width bmax.
__host__ __device__ inline uint32_t stage_bytes_for(uint32_t bmax) { return ((kWarpRows * bmax / 8 + 15) & ~15u) + 32; }

// ---------------------------------------------------------------- Fully-Parallel
// Extract and store the rows of a staged FOR/dictionary/Float2Int warp tile;
// returns true if a dictionary code was out of range or a Float2Int integer
// was beyond 2^53.
// FLOAT2INT (T = int64 bits of the doubles): the integer d = reference + u
// becomes the double nearest d / 10^e, built with integer multiplies
// (zf::f2i_bits; `e` and its reciprocal row `rr` are the chunk's).
// WIN: 1 = NARROW (b <= 8, four int32 values from one two-word window),
// 0 = one extraction per value, 2 = Float2Int chunk whose integers all lie in
// [0, 2^32) with e >= 1 (32-bit extraction and zf::f2i_bits_u32, `kexp` the
// chunk's exponent constant).
template <class T, int SCHEME, int WIN>
__device__ __forceinline__ bool fp_rows(const ZfDevChunk& c, const Hdr& h, T* dst, const uint32_t* wsm, uint32_t nr,
                                        uint32_t b, uint32_t lane, uint32_t e = 0,
                                        const zf::F2IRecip& rr = zf::F2IRecip{0, 0, 0, 0}, bool chk = true,
                                        int32_t kexp = 0) {
    // Float2Int: four values (a 32-byte sector) per lane per step
    constexpr int V = SCHEME == ZF_FLOAT2INT ? 4 : 16 / sizeof(T);
    const T* dict = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const T ref = (T)h.ref;
    const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    bool bad = false;
#pragma unroll 2
    for (uint32_t i0 = lane * V; i0 < nr; i0 += 32 * V) {
        if constexpr (WIN == 2) {
            const uint32_t m32 = b >= 32 ? 0xFFFFFFFFu : (1u << b) - 1u, ref32 = (uint32_t)h.ref;
            T v[V];
#pragma unroll
            for (int k = 0; k < V; k++) {
                const uint32_t pos = (i0 + k) * b, w = pos >> 5;
                const uint32_t u = __funnelshift_r(wsm[w], wsm[w + 1], pos & 31) & m32;
                v[k] = (T)zf::f2i_bits_u32(ref32 + u, e, rr, kexp);
            }
            if (i0 + V <= nr) {
                store_vec<T, V>(dst + i0, v, al32);
            } else {
#pragma unroll
                for (int k = 0; k < V; k++)
                    if (i0 + k < nr) dst[i0 + k] = v[k];
            }
            continue;
        }
        uint64_t u[V];
        if constexpr (WIN == 1 && V == 4) {
            uint32_t w4[4];
            extract4<true, uint32_t>(wsm, i0 * b, b, w4);
#pragma unroll
            for (int k = 0; k < V; k++) u[k] = w4[k];
        } else {
#pragma unroll
            for (int k = 0; k < V; k++) u[k] = extract(wsm, (i0 + k) * b, b);
        }
        T v[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            if constexpr (SCHEME == ZF_FOR_BP) {
                v[k] = (T)(ref + (T)u[k]);
            } else if constexpr (SCHEME == ZF_FLOAT2INT) {
                const int64_t d = (int64_t)(h.ref + u[k]);
                if (chk) bad |= i0 + k < nr && (d > zf::kF2IDMax || d < -zf::kF2IDMax);
                v[k] = (T)zf::f2i_bits(d, e, rr);
            } else {
                const bool in = i0 + k < nr;
                bad |= in && u[k] >= h.n_aux;
                v[k] = (in && u[k] < h.n_aux) ? __ldg(dict + u[k]) : (T)0;
            }
        }
        if (i0 + V <= nr) {
            store_vec<T, V>(dst + i0, v, al32);
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (i0 + k < nr) dst[i0 + k] = v[k];
        }
    }
    return bad;
}

// Float2Int exceptions of rows [r0, r0 + nrows): their rows are ascending,
// so a 32-way search (one load per lane per round) finds the first at or
// after r0, and the warp writes the stored 64 bits over the decoded rows.
__device__ __forceinline__ void f2i_exceptions(const ZfDevChunk& c, const Hdr& h, unsigned long long* dst,
                                               uint32_t r0, uint32_t nrows, uint32_t lane) {
    const uint32_t n = h.n_aux;
    if (n == 0) return;
    const uint32_t* pos = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const unsigned long long* val = reinterpret_cast<const unsigned long long*>(c.blob + h.off[2]);
    uint32_t lo = 0, hi = n;                      // rows at indices < lo are < r0; index hi counts as >= r0
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32, idx = lo + lane * step;
        const uint32_t ge = __ballot_sync(0xFFFFFFFFu, idx >= hi || __ldg(pos + idx) >= r0);
        if (ge & 1u) {
            hi = lo;
        } else {
            const uint32_t f = ge ? __ffs(ge) - 1 : 32;   // first sample at or after r0 (32: none)
            const uint32_t prev = lo + (f - 1) * step;
            hi = f < 32 ? min(hi, lo + f * step) : hi;
            lo = prev + 1;
        }
    }
    const uint32_t idx = lo + lane;
    const uint32_t ge = __ballot_sync(0xFFFFFFFFu, idx >= hi || __ldg(pos + idx) >= r0);
    uint32_t k0 = ge ? lo + __ffs(ge) - 1 : hi;
    __syncwarp();   // the decoded rows of this warp are written before they are replaced
    for (;; k0 += 32) {
        const uint32_t k = k0 + lane;
        const uint32_t r = k < n ? __ldg(pos + k) : 0xFFFFFFFFu;
        const bool in = r >= r0 && r - r0 < nrows;
        if (in) dst[r - r0] = __ldg(val + k);
        if (!__any_sync(0xFFFFFFFFu, in && k < n)) break;
    }
}

// SCHEME: ZF_FOR_BP, ZF_DICT_BP, ZF_FLOAT2INT or ZF_RAW.  Rows [r0, r0 + nrows)
// of the chunk (r0 a multiple of 1024).  The packed stream of consecutive
// tiles is contiguous, so tile i+1 is staged while tile i decodes.
template <class T, int SCHEME>
__device__ void fp_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                       uint32_t* err) {
    constexpr int V = 16 / sizeof(T);
    const uint32_t lane = threadIdx.x & 31;
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    if constexpr (SCHEME == ZF_RAW) {
        const T* src = reinterpret_cast<const T*>(c.blob + h.off[0]) + r0;
        for (uint32_t i0 = lane * V; i0 < nrows; i0 += 32 * V) {
            if (i0 + V <= nrows) reinterpret_cast<uint4*>(dst + i0)[0] = ldg16(src + i0);
            else
                for (uint32_t i = i0; i < nrows; i++) dst[i] = src[i];
        }
    } else {
        const uint32_t b = h.b;
        uint32_t e = 0;
        zf::F2IRecip rr{0, 0, 0, 0};
        bool chk = true;   // Float2Int: whether an integer of the chunk can pass 2^53
        bool u32 = false;  // Float2Int: e >= 1 and every integer of the chunk in [0, 2^32)
        if constexpr (SCHEME == ZF_FLOAT2INT) {
            e = c.blob[48];
            if (e > (uint32_t)zf::kF2IMaxExp) {
                if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
                return;
            }
            rr = kF2IRecip[e];
            const int64_t ref = (int64_t)h.ref;
            if (b <= 54 && ref >= -zf::kF2IDMax && ref <= zf::kF2IDMax)
                chk = ref + (int64_t)((1ull << b) - 1) > zf::kF2IDMax;
            u32 = e >= 1 && b <= 32 && ref >= 0 && ref + (int64_t)((1ull << b) - 1) < ((int64_t)1 << 32);
        }
        if (b > 8 * sizeof(T) || (SCHEME == ZF_DICT_BP && b > 16)) {
            if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
            return;
        }
        const uint8_t* sec = c.blob + h.off[SCHEME == ZF_DICT_BP ? 1 : 0];
        const uint32_t sb = stage_bytes_for(b) / 4;          // words per staging buffer
        const uint32_t ntiles = (nrows + kWarpRows - 1) / kWarpRows;
        auto issue = [&](uint32_t i) {
            const uint32_t rr = r0 + i * kWarpRows, nr = min(kWarpRows, r0 + nrows - rr);
            stage_async(wsm + (i & 1) * sb, sec + ((uint64_t)rr * b >> 3), (nr * b + 7) >> 3, lane);
            __pipeline_commit();
        };
        issue(0);
        bool bad = false;
        for (uint32_t i = 0; i < ntiles; i++) {
            if (i + 1 < ntiles) {
                issue(i + 1);
                __pipeline_wait_prior(1);
            } else {
                __pipeline_wait_prior(0);
            }
            __syncwarp();
            const uint32_t nr = min(kWarpRows, nrows - i * kWarpRows);
            const uint32_t* buf = wsm + (i & 1) * sb;
            if (V == 4 && b <= 8) bad |= fp_rows<T, SCHEME, 1>(c, h, dst + i * kWarpRows, buf, nr, b, lane);
            else if (SCHEME == ZF_FLOAT2INT && u32)
                fp_rows<T, SCHEME, 2>(c, h, dst + i * kWarpRows, buf, nr, b, lane, e, rr, false,
                                      1052 - (int32_t)rr.s - (int32_t)e);
            else bad |= fp_rows<T, SCHEME, 0>(c, h, dst + i * kWarpRows, buf, nr, b, lane, e, rr, chk);
            __syncwarp();
        }
        if (bad) report(err, ZF_ECORRUPT, c.chunk_id);
        if constexpr (SCHEME == ZF_FLOAT2INT)
            f2i_exceptions(c, h, reinterpret_cast<unsigned long long*>(dst), r0, nrows, lane);
    }
}

// ---------------------------------------------------------------- delta (Group-Parallel)
// Swizzle of the 16-byte chunks of a lane's 128-byte line in the transpose
// buffer: x = 4a + c (a < 2, c < 4) -> 2c + a.  Eight consecutive lanes
// writing chunk k land in eight different bank groups, and so do the eight
// lanes of a read phase (two lane quads reading the even or the odd chunks of
// owners 4 apart, whose swizzles differ in parity).
__device__ __forceinline__ uint32_t xswz(uint32_t l) {
    l &= 7;
    return ((l & 3) << 1) | (l >> 2);
}

// Stores of lane-owned lines, four lanes per line: every lane has put its
// 128-byte line (eight 16-byte chunks, swizzled) in `xb`; in step r the lanes
// of quad q write the four 32-byte sectors of lane 4q + r's line, so each
// 256-bit store instruction writes eight whole 128-byte lines instead of 32
// single sectors of 32 lines (the L2 takes a quarter of the requests).
// `line0` is lane 0's line; lane o's is line0 + o * lane_bytes.
__device__ __forceinline__ void store_lines_x4(char* line0, uint32_t lane_bytes, const uint4* xb, uint32_t lane) {
    const uint32_t q4 = lane & ~3u, i4 = lane & 3u;
#pragma unroll
    for (uint32_t r = 0; r < 4; r++) {
        const uint32_t o = q4 + r, fo = xswz(o);
        const uint4 a = xb[o * 8 + ((2 * i4) ^ fo)], c = xb[o * 8 + ((2 * i4 + 1) ^ fo)];
        store32(line0 + o * lane_bytes + 32 * i4, ((unsigned long long)a.y << 32) | a.x,
                ((unsigned long long)a.w << 32) | a.z, ((unsigned long long)c.y << 32) | c.x,
                ((unsigned long long)c.w << 32) | c.z);
    }
}

// One 1024-row block with each lane owning 32 consecutive values
// [32*lane, 32*lane + 32): a single warp scan per block.  The lane's bits
// start on a word boundary (32*lane*b bits = lane*b words), so every lane
// walks the same bit positions and the refill of the two-word bit reader is
// uniform across the warp.  The lane's differences are read twice: once for
// their sum (the warp scan needs it first), once to rebuild the values, so no
// array of prefixes stays live in registers.  Full blocks at a 32-byte
// aligned address leave through the transpose buffer `xb` (4 KiB per warp),
// four lanes per 128-byte line (store_lines_x4); other blocks in 32-byte
// stores (four int64 or eight int32), each a whole L2 sector.  WIDE
// (b > 21): 64-bit sums and funnel-shift extraction; otherwise 32-bit sums
// (32 * 1024 * (2^21 - 1) < 2^32).
template <class T, bool WIDE, bool WS>
__device__ __forceinline__ void delta_block_lanes(T* dst, const uint32_t* wsm, uint32_t mk, uint32_t b, uint64_t base,
                                                  uint64_t min_d, uint32_t lane, uint4* xb) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    using S = typename std::conditional<WIDE, unsigned long long, unsigned int>::type;
    constexpr int PER = 32 / sizeof(T);           // values per 32-byte store
    const uint32_t j0 = lane * 32;
    const uint32_t nv = mk > j0 ? min(32u, mk - j0) : 0u;   // valid values of this lane
    const uint32_t mask = WIDE ? 0u : (1u << b) - 1u;
    // bit reader over the lane's differences (narrow: two words in registers)
    uint32_t wi = 0, lo = 0, hi = 0, pos = 0;
    auto start = [&]() {
        if constexpr (!WIDE) {
            wi = lane * b;
            lo = wsm[wi];
            hi = wsm[wi + 1];
            wi += 2;
            pos = 0;
        }
    };
    // difference k of the lane (u_0 of the block and slots past the block count as 0)
    auto diff = [&](uint32_t k, bool full) -> S {
        S u;
        if constexpr (!WIDE) {
            u = __funnelshift_r(lo, hi, pos) & mask;
            pos += b;
            if (pos >= 32) {
                lo = hi;
                hi = wsm[wi++];
                pos -= 32;
            }
        } else {
            u = (full || k < nv) ? (S)extract(wsm, (j0 + k) * b, b) : (S)0;
        }
        if ((!full && k >= nv) || (k == 0 && lane == 0)) u = 0;
        return u;
    };
    start();
    S total = 0;
#pragma unroll
    for (uint32_t k = 0; k < 32; k++) total += diff(k, false);
    const S excl = warp_incl_sum<S>(total, lane) - total;
    const U md = (U)min_d;
    // x_{j0+k} = base + (j0 + k) * min_d + (differences up to j0 + k): acc after
    // step k, where each step adds min_d + u_k
    U acc = (U)base + (U)j0 * md + (U)excl - md;
    start();
    const bool al32 = WS && (reinterpret_cast<uintptr_t>(dst + j0) & 31) == 0;
    if constexpr (WS && !WIDE) {
        if (al32 && mk == zf::kDeltaBlock) {   // warp-uniform: dst is the block's first row
            constexpr uint32_t LANE_BYTES = 32 * sizeof(T), LINES = LANE_BYTES / 128;
            const uint32_t f = xswz(lane);
#pragma unroll
            for (uint32_t h = 0; h < LINES; h++) {
#pragma unroll
                for (uint32_t k8 = 0; k8 < 8; k8++) {
                    uint4 w;
                    if constexpr (sizeof(T) == 8) {
                        const uint32_t k = h * 16 + k8 * 2;
                        acc += md + (U)diff(k, true);
                        const U v0 = acc;
                        acc += md + (U)diff(k + 1, true);
                        w = make_uint4((uint32_t)v0, (uint32_t)(v0 >> 32), (uint32_t)acc, (uint32_t)(acc >> 32));
                    } else {
                        uint32_t a[4];
#pragma unroll
                        for (uint32_t e = 0; e < 4; e++) {
                            acc += md + (U)diff(k8 * 4 + e, true);
                            a[e] = (uint32_t)acc;
                        }
                        w = make_uint4(a[0], a[1], a[2], a[3]);
                    }
                    xb[lane * 8 + (k8 ^ f)] = w;
                }
                __syncwarp();
                store_lines_x4(reinterpret_cast<char*>(dst) + h * 128, LANE_BYTES, xb, lane);
                __syncwarp();
            }
            return;
        }
    }
#pragma unroll
    for (int q = 0; q < 32 / PER; q++) {
        T v[PER];
#pragma unroll
        for (int e = 0; e < PER; e++) {
            acc += md + (U)diff(q * PER + e, false);
            v[e] = (T)acc;
        }
        if ((uint32_t)(q * PER + PER) <= nv) {
            if (WS && al32) {
                if constexpr (sizeof(T) == 8) {
                    store32(dst + j0 + q * PER, (uint64_t)v[0], (uint64_t)v[1], (uint64_t)v[2], (uint64_t)v[3]);
                } else {
                    store32(dst + j0 + q * PER, ((uint64_t)(uint32_t)v[1] << 32) | (uint32_t)v[0],
                            ((uint64_t)(uint32_t)v[3] << 32) | (uint32_t)v[2],
                            ((uint64_t)(uint32_t)v[5] << 32) | (uint32_t)v[4],
                            ((uint64_t)(uint32_t)v[7] << 32) | (uint32_t)v[6]);
                }
            } else {
                store_vec<T, PER>(dst + j0 + q * PER, v);
            }
        } else {
#pragma unroll
            for (int e = 0; e < PER; e++)
                if ((uint32_t)(q * PER + e) < nv) dst[j0 + q * PER + e] = v[e];
        }
    }
}

// Blocks of more than 21 bits per difference are rare; out of line, they do
// not add to the registers of the common path.  They keep 16-byte stores: in
// an out-of-line function a 256-bit store from inline PTX wrote only part of
// its data (seen on GB300; the same store inlined is exact).
template <class T>
__device__ __noinline__ void delta_block_wide(T* dst, const uint32_t* wsm, uint32_t mk, uint32_t b, uint64_t base,
                                              uint64_t min_d, uint32_t lane) {
    delta_block_lanes<T, true, false>(dst, wsm, mk, b, base, min_d, lane, nullptr);
}

// Blocks of rows [r0, r0 + nrows) (r0 a multiple of 1024, at most 32 blocks).
// Lane j holds block j's 24-byte entry; block i+1's payload is staged while
// block i decodes.
template <class T, bool WS>
__device__ void delta_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                          uint32_t* err, uint32_t bmax) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t blk0 = r0 / zf::kDeltaBlock;
    const uint32_t nblk = (nrows + zf::kDeltaBlock - 1) / zf::kDeltaBlock;
    uint64_t e_base = 0, e_md = 0;
    uint32_t e_poff = 0, e_b = 0;
    if (lane < nblk) {
        const uint8_t* e = c.blob + h.off[0] + (uint64_t)(blk0 + lane) * zf::kDeltaEntry;
        const uint2 e0 = __ldg(reinterpret_cast<const uint2*>(e));
        const uint2 e1 = __ldg(reinterpret_cast<const uint2*>(e + 8));
        const uint2 e2 = __ldg(reinterpret_cast<const uint2*>(e + 16));
        e_base = ((uint64_t)e0.y << 32) | e0.x;
        e_md = ((uint64_t)e1.y << 32) | e1.x;
        e_poff = e2.x;
        e_b = e2.y & 0xFF;
    }
    // a block whose entry is inconsistent is reported and skipped
    const uint32_t mk_lane = min(zf::kDeltaBlock, nrows - min(nrows, lane * zf::kDeltaBlock));
    const bool lane_ok = lane >= nblk || (e_b <= 8 * sizeof(T) && e_b <= bmax && !(e_poff & 15) &&
                                          (uint64_t)e_poff + ((mk_lane * e_b + 7) >> 3) <= h.len[1]);
    const uint32_t ok_mask = __ballot_sync(0xFFFFFFFFu, lane_ok);
    if (ok_mask != 0xFFFFFFFFu && lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
    const uint32_t sb = stage_bytes_for(bmax) / 4;
    const uint8_t* payload = c.blob + h.off[1];
    auto issue = [&](uint32_t i) {
        const uint32_t poff = __shfl_sync(0xFFFFFFFFu, e_poff, i);
        const uint32_t b = __shfl_sync(0xFFFFFFFFu, e_b, i);
        const uint32_t mk = min(zf::kDeltaBlock, nrows - i * zf::kDeltaBlock);
        if ((ok_mask >> i) & 1) stage_async(wsm + (i & 1) * sb, payload + poff, (mk * b + 7) >> 3, lane);
        __pipeline_commit();
    };
    issue(0);
    for (uint32_t i = 0; i < nblk; i++) {
        if (i + 1 < nblk) {
            issue(i + 1);
            __pipeline_wait_prior(1);
        } else {
            __pipeline_wait_prior(0);
        }
        __syncwarp();
        const uint64_t base = __shfl_sync(0xFFFFFFFFu, e_base, i);
        const uint64_t md = __shfl_sync(0xFFFFFFFFu, e_md, i);
        const uint32_t b = __shfl_sync(0xFFFFFFFFu, e_b, i);
        const uint32_t mk = min(zf::kDeltaBlock, nrows - i * zf::kDeltaBlock);
        if ((ok_mask >> i) & 1) {
            T* dst = reinterpret_cast<T*>(c.dst) + r0 + i * zf::kDeltaBlock;
            const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
            const uint32_t* buf = wsm + (i & 1) * sb;
            uint4* xb = reinterpret_cast<uint4*>(wsm + 2 * sb);
            if (b <= 21) delta_block_lanes<T, false, WS>(dst, buf, mk, b, base, md, lane, xb);
            else delta_block_wide<T>(dst, buf, mk, b, base, md, lane);
            (void)al32;
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- RLE (Group-Parallel)
// Expansion of one 1024-row tile whose runs [rf, rf+m) have their lengths at
// `lens_al` + sft, lens_al 16-byte aligned and sft = rf mod 4 (staged in shared
// memory, or in global memory when the tile has more runs than a staging
// buffer holds), and their values at `vals`.  `bm` is the warp's 32-word
// bitmask of the tile's rows.
template <class T, bool WS>
__device__ __forceinline__ void rle_rows(const ZfDevChunk& c, const Hdr& h, T* dst, const uint32_t* lens_al,
                                         uint32_t sft, const T* vals, uint32_t* bm, uint32_t m, uint32_t skip,
                                         uint32_t nr, bool last_tile, uint32_t next_skip, uint32_t lane,
                                         uint32_t* err) {
    bm[lane] = 0;
    __syncwarp();
    // presum, 128 length entries per step: lane l reads entries 4l..4l+3 with
    // one 16-byte load (entry sft is the tile's first run), one warp scan of
    // the lanes' sums gives each run its start row relative to the first
    // run's start, and every run but the first sets the bit of its start row.
    // The tile's runs lie inside the chunk, so their lengths add up to at most
    // its rows (<= 2^30); sums saturate at kCap = 2^30 + 1, which no valid
    // tile reaches, so a stream whose lengths would wrap 32 bits is caught.
    constexpr uint32_t kCap = (1u << 30) + 1u;
    bool bad = false;
    uint32_t end = 0;                 // rows covered so far, counted from the first run's start
    uint32_t first_len = 0, my_last = 0;
    const uint32_t n = sft + m;       // entries from the aligned start
    for (uint32_t g = 0; g < n; g += 128) {
        const uint32_t k0 = g + 4 * lane;
        const uint4 q = k0 < n ? reinterpret_cast<const uint4*>(lens_al)[k0 >> 2] : make_uint4(0, 0, 0, 0);
        uint32_t L[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const uint32_t k = k0 + e;
            const bool valid = k >= sft && k < n;
            if (!valid) L[e] = 0;
            bad |= valid && (L[e] == 0 || L[e] > h.rows);
        }
        const uint32_t s4 = min(min(L[0] + L[1], kCap) + min(L[2] + L[3], kCap), kCap);
        const uint32_t incl = warp_incl_sum_sat(s4, kCap, lane);
        uint32_t st = end + incl - s4;  // start of entry k0
        // the lane's start bits, ORed per bitmask word in registers first (its
        // runs are consecutive, so their words are nondecreasing): one shared
        // atomic per word the lane touches instead of one per run
        uint32_t cw = 0xFFFFFFFFu, cbits = 0;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const uint32_t k = k0 + e;
            if (k > sft && k < n && st >= skip && st - skip < nr) {
                const uint32_t r = st - skip;
                if ((r >> 5) != cw) {
                    if (cbits) atomicOr(&bm[cw], cbits);
                    cw = r >> 5;
                    cbits = 0;
                }
                cbits |= 1u << (r & 31);
            }
            if (k + 1 == n) my_last = st;
            st += L[e];
        }
        if (cbits) atomicOr(&bm[cw], cbits);
        if (g == 0) {
            const uint32_t f0 = sft == 0 ? L[0] : sft == 1 ? L[1] : sft == 2 ? L[2] : L[3];
            first_len = __shfl_sync(0xFFFFFFFFu, f0, 0);   // run 0: entry sft of lane 0
        }
        end = min(end + __shfl_sync(0xFFFFFFFFu, incl, 31), kCap);
        if (end > h.rows) bad = true;
    }
    const uint32_t last_start = __shfl_sync(0xFFFFFFFFu, my_last, ((n - 1) & 127) >> 2);
    // The runs cover exactly [0, nr): the first starts at or before row 0, the
    // last ends at nr or continues into the next tile by the directory's amount.
    bool ok = skip < first_len && end >= skip;
    if (last_tile || next_skip == 0) ok &= end - skip == nr;
    else ok &= last_start - skip + next_skip == nr && end - skip > nr;
    const bool any_bad = __any_sync(0xFFFFFFFFu, bad);
    if (lane == 0 && (!ok || any_bad)) report(err, ZF_ECORRUPT, c.chunk_id);
    __syncwarp();
    // A row's run (relative to the tile's first) is the number of run starts
    // at or before it: lane l holds word l of the bitmask and the starts in
    // the words before it (one shuffle scan of the popcounts).  Expansion, 256
    // rows per step: lane l takes rows 8l..8l+7, a quarter of one word.  Each
    // run sets at most one bit and the first sets none, so a count never
    // passes m - 1.
    const uint32_t word = bm[lane];
    const uint32_t cnt = __popc(word);
    const uint32_t before = warp_incl_sum<uint32_t>(cnt, lane) - cnt;
    constexpr int V = 8;
    const bool al32 = WS && (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    const uint32_t o = (lane & 3) * 8;
    for (uint32_t row = 0; row * 256 < nr; row++) {
        const uint32_t j = row * 256 + lane * V;
        const uint32_t w = row * 8 + (lane >> 2);
        const uint32_t ww = __shfl_sync(0xFFFFFFFFu, word, w);
        uint32_t idx = __shfl_sync(0xFFFFFFFFu, before, w) + __popc(ww & ((1u << o) - 1u));
        const uint32_t b8 = ww >> o;
        T v[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            idx += (b8 >> k) & 1u;
            v[k] = vals[idx];
        }
        if (j + V <= nr) {
            if constexpr (sizeof(T) == 4) {
                store_vec<T, V>(dst + j, v, al32);
            } else {
                const T a[4] = {v[0], v[1], v[2], v[3]}, z[4] = {v[4], v[5], v[6], v[7]};
                store_vec<T, 4>(dst + j, a, al32);
                store_vec<T, 4>(dst + j + 4, z, al32);
            }
        } else {
#pragma unroll
            for (int k = 0; k < V; k++)
                if (j + k < nr) dst[j + k] = v[k];
        }
    }
    __syncwarp();
}

constexpr uint32_t kRleStageRuns = 256;   // runs per staging buffer
constexpr uint32_t kRleStages = 2;        // staging buffers per warp: tile i+1 loads while tile i expands

// Shared memory of one RLE staging buffer: lengths then values, each with
// room for the 16-byte aligned copy that starts up to 3 entries early.
__host__ __device__ inline uint32_t rle_buf_bytes(uint32_t value_bytes) {
    return (kRleStageRuns + 4) * 4 + (((kRleStageRuns + 4) * value_bytes + 15) & ~15u);
}

// Tiles of rows [r0, r0 + nrows) (r0 a multiple of 1024, at most 31 tiles).
// Lane j holds the directory entry of tile j (and of the tile after the
// last); the next tile's lengths and values are staged while a tile expands.
template <class T, bool WS>
__device__ void rle_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                        uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    if (h.rows > (1u << 30)) {   // chunks hold at most 2^30 rows (the presum relies on it)
        if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const T* vals = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const uint32_t* lens = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const uint2* dir = reinterpret_cast<const uint2*>(c.blob + h.off[2]);
    const uint32_t R = h.n_aux;
    const uint32_t t0 = r0 / zf::kRleDirRows;
    const uint32_t nt = (nrows + zf::kRleDirRows - 1) / zf::kRleDirRows;
    const uint32_t tiles_in_chunk = (h.rows + zf::kRleDirRows - 1) / zf::kRleDirRows;
    uint2 d = make_uint2(0, 0);
    if (lane <= nt && t0 + lane < tiles_in_chunk) d = __ldg(dir + t0 + lane);
    uint32_t* bm = wsm;
    uint8_t* bufs = reinterpret_cast<uint8_t*>(wsm) + 128;
    const uint32_t bb = rle_buf_bytes(sizeof(T));
    constexpr uint32_t VPER = 16 / sizeof(T);   // values per 16-byte copy
    // run range [rf, rf + m) of tile i, or m = 0 if its directory entries are inconsistent
    auto runs = [&](uint32_t i, uint32_t& rf, uint32_t& skip, uint32_t& m, uint32_t& next_skip, bool& last) {
        rf = __shfl_sync(0xFFFFFFFFu, d.x, i);
        skip = __shfl_sync(0xFFFFFFFFu, d.y, i);
        const uint32_t nx = __shfl_sync(0xFFFFFFFFu, d.x, i + 1);
        next_skip = __shfl_sync(0xFFFFFFFFu, d.y, i + 1);
        const uint32_t rr = r0 + i * zf::kRleDirRows, nr = min(zf::kRleDirRows, r0 + nrows - rr);
        last = rr + nr >= h.rows;
        uint32_t rl = R - 1;
        bool bad = (rr == 0 && (rf != 0 || skip != 0)) || R == 0 || skip >= h.rows;
        if (!last) {
            bad |= next_skip == 0 && nx == 0;
            rl = next_skip > 0 ? nx : nx - 1;
        } else {
            next_skip = 0;
        }
        bad |= rf > rl || rl >= R || rl - rf + 1 > nr + 1;
        m = bad ? 0 : rl - rf + 1;
    };
    auto issue = [&](uint32_t i) {
        uint32_t rf, skip, m, ns;
        bool last;
        runs(i, rf, skip, m, ns, last);
        if (m && m <= kRleStageRuns) {
            // 16-byte copies from the aligned entries at or before rf (the
            // sections are 16-byte aligned and padded, so they stay inside)
            uint8_t* b = bufs + (i % kRleStages) * bb;
            const uint32_t l0 = rf & ~3u, nl = (rf + m - l0 + 3) / 4;
            const uint32_t v0 = rf & ~(VPER - 1), nv = (rf + m - v0 + VPER - 1) / VPER;
            for (uint32_t k = lane; k < nl; k += 32)
                __pipeline_memcpy_async(b + 16 * k, lens + l0 + 4 * k, 16);
            for (uint32_t k = lane; k < nv; k += 32)
                __pipeline_memcpy_async(b + (kRleStageRuns + 4) * 4 + 16 * k, vals + v0 + VPER * k, 16);
        }
        __pipeline_commit();
    };
    // The next kRleStages - 1 tiles are staged while a tile expands (one
    // commit group per tile, empty ones included).  Deeper staging (four
    // buffers) measured slower on GB300: it costs occupancy.
    for (uint32_t i = 0; i + 1 < kRleStages && i < nt; i++) issue(i);
    for (uint32_t i = 0; i < nt; i++) {
        if (i + kRleStages - 1 < nt) issue(i + kRleStages - 1);
        switch (min(nt - 1, i + kRleStages - 1) - i) {   // groups committed after tile i's
        case 0: __pipeline_wait_prior(0); break;
        case 1: __pipeline_wait_prior(1); break;
        case 2: __pipeline_wait_prior(2); break;
        default: __pipeline_wait_prior(3); break;
        }
        __syncwarp();
        uint32_t rf, skip, m, ns;
        bool last;
        runs(i, rf, skip, m, ns, last);
        const uint32_t rr = r0 + i * zf::kRleDirRows, nr = min(zf::kRleDirRows, r0 + nrows - rr);
        if (!m) {
            if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        } else {
            T* dst = reinterpret_cast<T*>(c.dst) + rr;
            if (m <= kRleStageRuns) {
                const uint8_t* b = bufs + (i % kRleStages) * bb;
                rle_rows<T, WS>(c, h, dst, reinterpret_cast<const uint32_t*>(b), rf & 3u,
                                reinterpret_cast<const T*>(b + (kRleStageRuns + 4) * 4) + (rf & (VPER - 1)), bm, m,
                                skip, nr, last, ns, lane, err);
            } else {
                rle_rows<T, WS>(c, h, dst, lens + (rf & ~3u), rf & 3u, vals + rf, bm, m, skip, nr, last, ns, lane,
                                err);
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------- string dictionary sizes
// (the decoder is in zf_strdict.cuh)
constexpr uint32_t kStrCodeBuf = (1024u * 16u / 8u) + 32u;   // one tile of codes at b <= 16, plus the reader's overrun
constexpr uint32_t kStrWin = 16u * zf::kStrTokenMax + 32u;    // 16 tokens of at most 64 bytes, at the output's alignment

// ---------------------------------------------------------------- single-tile entry points
// (used by the allocation-free kernel; 16-byte stores only)
template <class T, int SCHEME>
__device__ __forceinline__ void fp_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* wsm,
                                        uint32_t* err) {
    fp_job<T, SCHEME>(c, h, r0, nr, wsm, err);
}
template <class T>
__device__ __forceinline__ void delta_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr,
                                           uint32_t* wsm, uint32_t* err) {
    delta_job<T, false>(c, h, r0, nr, wsm, err, 8 * sizeof(T));
}
template <class T>
__device__ __forceinline__ void rle_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* wsm,
                                         uint32_t* err) {
    rle_job<T, false>(c, h, r0, nr, wsm, err);
}

// Shared memory (bytes) one warp needs for a scheme, given the value size and
// the widest bit width of the chunks it decodes (two staging buffers).
__host__ __device__ inline uint32_t warp_smem(int scheme, uint32_t value_bytes, uint32_t bmax) {
    switch (scheme) {
    case ZF_FOR_BP: case ZF_DICT_BP: case ZF_FLOAT2INT: return 2 * stage_bytes_for(bmax);
    case ZF_DELTA_BP: return 2 * stage_bytes_for(bmax) + 4096;   // + the store transpose buffer
    case ZF_RLE: return 128 + kRleStages * rle_buf_bytes(value_bytes);   // row bitmask + staging buffers
    case ZF_STRDICT: return kStrCodeBuf + kStrWin;                      // one tile of codes + the output window
    }
    return 0;
}

}  // namespace zfd
