// zf_device.cuh -- device-side decode of one warp tile (1024 output rows) of
// one chunk, per scheme.
//
// A launch decodes a list of chunks (ZfDevChunk).  A CTA takes a CTA tile of
// `tile_rows` rows of one chunk; each of its warps decodes 1024-row warp
// tiles of it on its own, with its own slice of shared memory and no
// CTA-wide barrier, so an SM keeps dozens of independent warp tiles in
// flight.  The decoders follow the parallel patterns of Section 3.1:
//   fp_warp     Fully-Parallel: FOR / dictionary / raw.  The warp stages the
//               tile's packed words in shared memory with coalesced 16-byte
//               loads, then every lane extracts C = 16/sizeof(T) consecutive
//               values with funnel shifts and writes them with one 16-byte
//               store (128 or 64 rows per warp step, coalesced).
//   delta_warp  Group-Parallel: one 1024-row delta block per warp tile, in
//               rows of 128 values: 4 per lane, a lane-local prefix, a warp
//               shuffle scan, and base + j*min_d added on the way out.
//   rle_warp    Group-Parallel: the tile's runs (the chunk's 1024-row
//               directory names the first) have their lengths scanned by warp
//               shuffles into start rows (the presum of Section 3.2); each run
//               start marks its row in shared memory and a running max over
//               the rows gives every row its run.  Each tile writes exactly
//               1024 rows, so long and short runs balance.
// A failed check of the stream sets a bit in the launch's error word; the
// tile then writes in-bounds placeholder values.  Nothing traps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "zf_internal.h"

namespace zfd {

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

// The warp copies `nbytes` from a 16-byte aligned global address into its
// shared-memory slice, 16 bytes per lane per step, then zeroes 32 bytes after.
__device__ __forceinline__ void warp_stage(uint32_t* wsm, const uint8_t* src, uint32_t nbytes, uint32_t lane) {
    uint32_t nvec = (nbytes + 15) >> 4;
    uint4* s4 = reinterpret_cast<uint4*>(wsm);
    for (uint32_t i = lane; i < nvec; i += 32) s4[i] = ldg16(src + 16ull * i);
    if (lane < 2) s4[nvec + lane] = make_uint4(0, 0, 0, 0);
    __syncwarp();
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
            ulonglong4_32a q;
            q.x = ((unsigned long long)w[1] << 32) | w[0];
            q.y = ((unsigned long long)w[3] << 32) | w[2];
            q.z = ((unsigned long long)w[5] << 32) | w[4];
            q.w = ((unsigned long long)w[7] << 32) | w[6];
            *reinterpret_cast<ulonglong4_32a*>(dst) = q;
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

__device__ __forceinline__ uint32_t warp_incl_max(uint32_t x, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x = max(x, y);
    }
    return x;
}

// ---------------------------------------------------------------- Fully-Parallel
template <bool NARROW, class S>
__device__ __forceinline__ void extract4(const uint32_t* wsm, uint32_t bitpos, uint32_t b, S (&u)[4]);

// Extract and store the rows of a staged FOR/dictionary warp tile; returns
// true if a dictionary code was out of range.
template <class T, int SCHEME, bool NARROW>
__device__ __forceinline__ bool fp_rows(const ZfDevChunk& c, const Hdr& h, T* dst, const uint32_t* wsm, uint32_t nr,
                                        uint32_t b, uint32_t lane) {
    constexpr int V = 16 / sizeof(T);
    const T* dict = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const T ref = (T)h.ref;
    bool bad = false;
#pragma unroll 2
    for (uint32_t i0 = lane * V; i0 < nr; i0 += 32 * V) {
        uint64_t u[V];
        if constexpr (NARROW && V == 4) {
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
            } else {
                bad |= u[k] >= h.n_aux;
                v[k] = u[k] < h.n_aux ? __ldg(dict + u[k]) : (T)0;
            }
        }
        if (i0 + V <= nr) store_vec<T, V>(dst + i0, v);
        else
            for (uint32_t i = i0; i < nr; i++) dst[i] = v[i - i0];
    }
    return bad;
}

// SCHEME: ZF_FOR_BP, ZF_DICT_BP or ZF_RAW.  Rows [r0, r0+nr) of the chunk, nr <= 1024.
template <class T, int SCHEME>
__device__ void fp_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* wsm,
                        uint32_t* err) {
    constexpr int V = 16 / sizeof(T);
    const uint32_t lane = threadIdx.x & 31;
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    if constexpr (SCHEME == ZF_RAW) {
        const T* src = reinterpret_cast<const T*>(c.blob + h.off[0]) + r0;
        for (uint32_t i0 = lane * V; i0 < nr; i0 += 32 * V) {
            if (i0 + V <= nr) reinterpret_cast<uint4*>(dst + i0)[0] = ldg16(src + i0);
            else
                for (uint32_t i = i0; i < nr; i++) dst[i] = src[i];
        }
    } else {
        const uint32_t b = h.b;
        if (b > 8 * sizeof(T) || (SCHEME == ZF_DICT_BP && b > 16)) {
            if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
            return;
        }
        const uint8_t* sec = c.blob + h.off[SCHEME == ZF_DICT_BP ? 1 : 0];
        warp_stage(wsm, sec + ((uint64_t)r0 * b >> 3), (nr * b + 7) >> 3, lane);
        bool bad;
        if (V == 4 && b <= 8) bad = fp_rows<T, SCHEME, true>(c, h, dst, wsm, nr, b, lane);
        else bad = fp_rows<T, SCHEME, false>(c, h, dst, wsm, nr, b, lane);
        if (bad) report(err, ZF_ECORRUPT, c.chunk_id);
        __syncwarp();
    }
}

// ---------------------------------------------------------------- delta (Group-Parallel)
// One 1024-row block: x_j = base + j*min_d + sum_{k=1..j} u_k (mod 2^width).
// Four consecutive b-bit values starting at bit `bitpos`.  WIDE = false needs
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

template <class T, class S, bool NARROW>
__device__ __forceinline__ void delta_rows(T* dst, const uint32_t* wsm, uint32_t mk, uint32_t b, uint64_t base,
                                           uint64_t min_d, uint32_t lane, bool al32) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    U acc = 0;
    const U md = (U)min_d;
    U t = (U)base + (U)(lane * 4) * md;          // base + j0 * min_d, advanced by 128 * min_d per row
    const U row_step = (U)128 * md;
    for (uint32_t row = 0; row * 128 < mk; row++) {
        const uint32_t j0 = row * 128 + lane * 4;
        S u[4];
        extract4<NARROW, S>(wsm, j0 * b, b, u);
        if (j0 == 0) u[0] = 0;                    // slot 0 carries no difference
        if (j0 + 4 > mk) {
#pragma unroll
            for (int k = 0; k < 4; k++)
                if (j0 + k >= mk) u[k] = 0;
        }
        S s1 = u[0] + u[1], s2 = s1 + u[2], s3 = s2 + u[3];
        S incl = warp_incl_sum<S>(s3, lane);
        S tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        U x0 = t + acc + (U)(incl - s3) + (U)u[0];
        T out[4];
        out[0] = (T)x0;
        out[1] = (T)(x0 + md + (U)(s1 - u[0]));
        out[2] = (T)(x0 + 2 * md + (U)(s2 - u[0]));
        out[3] = (T)(x0 + 3 * md + (U)(s3 - u[0]));
        if (j0 + 4 <= mk) store_vec<T, 4>(dst + j0, out, al32);
        else
            for (uint32_t k = 0; j0 + k < mk; k++) dst[j0 + k] = out[k];
        acc += (U)tot;
        t += row_step;
    }
}

// b <= 8: two rows of 128 values per step.  A lane's four differences sum to
// at most 4 * 255 and a row to at most 32,640 < 2^16, so both rows' lane sums
// share one 32-bit word (row a low, row b high) and one shuffle scan.
template <class T>
__device__ __forceinline__ void delta_rows_pair(T* dst, const uint32_t* wsm, uint32_t mk, uint32_t b, uint64_t base,
                                                uint64_t min_d, uint32_t lane, bool al32) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    U acc = 0;
    const U md = (U)min_d;
    U t = (U)base + (U)(lane * 4) * md;
    const U row_step = (U)128 * md;
    for (uint32_t row = 0; row * 128 < mk; row += 2) {
        const uint32_t ja = row * 128 + lane * 4, jb = ja + 128;
        uint32_t ua[4], ub[4];
        extract4<true, uint32_t>(wsm, ja * b, b, ua);
        extract4<true, uint32_t>(wsm, jb * b, b, ub);
        if (ja == 0) ua[0] = 0;
        if (jb + 4 > mk) {
#pragma unroll
            for (int k = 0; k < 4; k++) {
                if (ja + k >= mk) ua[k] = 0;
                if (jb + k >= mk) ub[k] = 0;
            }
        }
        const uint32_t a1 = ua[0] + ua[1], a2 = a1 + ua[2], a3 = a2 + ua[3];
        const uint32_t b1 = ub[0] + ub[1], b2 = b1 + ub[2], b3 = b2 + ub[3];
        const uint32_t packed = a3 | (b3 << 16);
        const uint32_t incl = warp_incl_sum<uint32_t>(packed, lane);
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const uint32_t excl = incl - packed;
        const U xa = t + acc + (U)(excl & 0xFFFFu) + (U)ua[0];
        const U xb = t + row_step + acc + (U)(tot & 0xFFFFu) + (U)(excl >> 16) + (U)ub[0];
        T oa[4], ob[4];
        oa[0] = (T)xa;
        oa[1] = (T)(xa + md + (U)(a1 - ua[0]));
        oa[2] = (T)(xa + 2 * md + (U)(a2 - ua[0]));
        oa[3] = (T)(xa + 3 * md + (U)(a3 - ua[0]));
        ob[0] = (T)xb;
        ob[1] = (T)(xb + md + (U)(b1 - ub[0]));
        ob[2] = (T)(xb + 2 * md + (U)(b2 - ub[0]));
        ob[3] = (T)(xb + 3 * md + (U)(b3 - ub[0]));
        if (ja + 4 <= mk) store_vec<T, 4>(dst + ja, oa, al32);
        else
            for (uint32_t k = 0; ja + k < mk; k++) dst[ja + k] = oa[k];
        if (jb + 4 <= mk) store_vec<T, 4>(dst + jb, ob, al32);
        else
            for (uint32_t k = 0; jb + k < mk; k++) dst[jb + k] = ob[k];
        acc += (U)(tot & 0xFFFFu) + (U)(tot >> 16);
        t += 2 * row_step;
    }
}

template <class T>
__device__ void delta_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* wsm,
                           uint32_t* err) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t blk = r0 / zf::kDeltaBlock;
    const uint8_t* e = c.blob + h.off[0] + (uint64_t)blk * zf::kDeltaEntry;
    // 24-byte entry: base, min_d, payload offset, b (8-byte aligned)
    uint2 e0 = __ldg(reinterpret_cast<const uint2*>(e));
    uint2 e1 = __ldg(reinterpret_cast<const uint2*>(e + 8));
    uint2 e2 = __ldg(reinterpret_cast<const uint2*>(e + 16));
    uint64_t base = ((uint64_t)e0.y << 32) | e0.x;
    uint64_t min_d = ((uint64_t)e1.y << 32) | e1.x;
    uint32_t poff = e2.x, b = e2.y & 0xFF;
    uint32_t nbytes = (nr * b + 7) >> 3;
    if (b > 8 * sizeof(T) || (poff & 15) || (uint64_t)poff + nbytes > h.len[1] || nr > zf::kDeltaBlock) {
        if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    warp_stage(wsm, c.blob + h.off[1] + poff, nbytes, lane);
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    // 128 values of at most 24 bits sum below 2^31: scan in 32 bits
    if (b <= 8) delta_rows_pair<T>(dst, wsm, nr, b, base, min_d, lane, al32);
    else if (b <= 24) delta_rows<T, uint32_t, false>(dst, wsm, nr, b, base, min_d, lane, al32);
    else delta_rows<T, U, false>(dst, wsm, nr, b, base, min_d, lane, al32);
    __syncwarp();
}

// ---------------------------------------------------------------- RLE (Group-Parallel)
// The warp's slice holds one u16 per row -- the index (relative to the tile's
// first run) of a run that starts at that row, 0 elsewhere -- followed by the
// values of the tile's runs.
template <class T>
__device__ void rle_warp(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* wsm,
                         uint32_t* err) {
    constexpr int V = 4;
    const uint32_t lane = threadIdx.x & 31;
    const T* vals = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const uint32_t* lens = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const uint2* dir = reinterpret_cast<const uint2*>(c.blob + h.off[2]);
    const uint32_t R = h.n_aux;
    const uint32_t t = r0 / zf::kRleDirRows;
    const uint2 e0 = __ldg(dir + t);
    const uint32_t rf = e0.x, skip = e0.y;
    const bool last_tile = r0 + nr >= h.rows;
    uint32_t rl = R - 1, next_skip = 0;
    bool bad = false;
    if (!last_tile) {
        const uint2 e1 = __ldg(dir + t + 1);
        next_skip = e1.y;
        bad |= e1.y == 0 && e1.x == 0;
        rl = e1.y > 0 ? e1.x : e1.x - 1;
    }
    bad |= r0 == 0 && (rf != 0 || skip != 0);
    if (bad || R == 0 || rf > rl || rl >= R || rl - rf + 1 > nr + 1 || nr > zf::kRleDirRows || skip >= h.rows) {
        if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t m = rl - rf + 1;
    uint16_t* mark = reinterpret_cast<uint16_t*>(wsm);
    T* rv = reinterpret_cast<T*>(wsm + zf::kRleDirRows / 2);
#pragma unroll
    for (int q = 0; q < 4; q++) reinterpret_cast<uint4*>(mark)[lane + 32 * q] = make_uint4(0, 0, 0, 0);
    __syncwarp();
    // presum: start row of each run relative to the tile, 32 runs per step.
    // Lengths are at most the chunk's rows (< 2^30), and only the first and
    // last run of a tile can be longer than the tile, so 32-bit sums hold.
    uint32_t end = 0;                 // rows covered so far, counted from the first run's start
    uint32_t first_len = 0, last_start = 0;
    for (uint32_t g0 = 0; g0 < m; g0 += 128) {
        // four groups of 32 runs: independent loads first, then the scans
        uint32_t Ls[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t i = g0 + 32 * q + lane;
            Ls[q] = 0;
            if (i < m) {
                Ls[q] = __ldg(lens + rf + i);
                rv[i] = __ldg(vals + rf + i);
            }
        }
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const uint32_t g = g0 + 32 * q;
            if (g >= m) break;
            const uint32_t i = g + lane;
            const uint32_t L = Ls[q];
            bad |= i < m && (L == 0 || L > h.rows);
            const uint32_t incl = warp_incl_sum<uint32_t>(L, lane);
            const uint32_t start = end + incl - L;   // relative to the first run's start
            if (i < m && i > 0 && start >= skip && start - skip < nr) mark[start - skip] = (uint16_t)i;
            if (g == 0) first_len = __shfl_sync(0xFFFFFFFFu, L, 0);
            const uint32_t ls = __shfl_sync(0xFFFFFFFFu, start, (m - 1 - g) & 31);
            if (m - 1 - g < 32) last_start = ls;
            end += __shfl_sync(0xFFFFFFFFu, incl, 31);
            if (end > 2u * (1u << 30) + 2048u) bad = true;
        }
    }
    // The runs cover exactly [0, nr): the first starts at or before row 0, the
    // last ends at nr or continues into the next tile by the directory's amount.
    bool ok = skip < first_len && end >= skip;
    if (last_tile || next_skip == 0) ok &= end - skip == nr;
    else ok &= last_start - skip + next_skip == nr && end - skip > nr;
    const bool any_bad = __any_sync(0xFFFFFFFFu, bad);
    if (lane == 0 && (!ok || any_bad)) report(err, ZF_ECORRUPT, c.chunk_id);
    __syncwarp();
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    uint32_t carry = 0;
    for (uint32_t j0 = lane * V; j0 - lane * V < nr; j0 += 32 * V) {
        const uint2 mk = reinterpret_cast<const uint2*>(mark)[j0 / 4];
        uint32_t r[V];
        r[0] = mk.x & 0xFFFF;
        r[1] = max(r[0], mk.x >> 16);
        r[2] = max(r[1], mk.y & 0xFFFF);
        r[3] = max(r[2], mk.y >> 16);
        const uint32_t incl = warp_incl_max(r[3], lane);
        uint32_t before = __shfl_up_sync(0xFFFFFFFFu, incl, 1);
        before = lane ? max(before, carry) : carry;
        T v[V];
#pragma unroll
        for (int k = 0; k < V; k++) v[k] = rv[min(max(before, r[k]), m - 1)];
        if (j0 + V <= nr) store_vec<T, V>(dst + j0, v, al32);
        else
            for (uint32_t k = 0; j0 + k < nr; k++) dst[j0 + k] = v[k];
        carry = max(carry, __shfl_sync(0xFFFFFFFFu, incl, 31));
    }
    __syncwarp();
}

// Shared memory (bytes) one warp needs for a scheme, given the value size and
// the widest bit width of the chunks it decodes.
__host__ __device__ inline uint32_t warp_smem(int scheme, uint32_t value_bytes, uint32_t bmax) {
    switch (scheme) {
    case ZF_FOR_BP: case ZF_DICT_BP: case ZF_DELTA_BP: return ((kWarpRows * bmax / 8 + 15) & ~15u) + 32;
    case ZF_RLE: return kWarpRows * 2 + (((kWarpRows + 1) * value_bytes + 15) & ~15u);  // marks + run values
    }
    return 0;
}

}  // namespace zfd
