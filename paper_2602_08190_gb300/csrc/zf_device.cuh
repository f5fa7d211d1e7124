// zf_device.cuh -- device-side decode of one tile of one chunk, per scheme.
//
// A launch decodes a list of chunks (ZfDevChunk) cut into tiles of
// `tile_rows` output rows.  Each CTA decodes whole tiles; the functions here
// decode one tile with all threads of the CTA.  They follow the parallel
// patterns of Section 3.1:
//   fp_tile     Fully-Parallel: FOR / dictionary / raw.  The tile's packed
//               words are staged in shared memory with 16-byte loads, then
//               every thread extracts C = 16/sizeof(T) consecutive values with
//               funnel shifts and writes them with one 16-byte store.
//   delta_tile  Group-Parallel: one 1024-row block at a time, thread-local
//               sums, a CTA-wide prefix scan (warp shuffles), base + j*min_d.
//   rle_tile    Group-Parallel: the tile's runs (found through the chunk's
//               1024-row directory) are loaded to shared memory, their lengths
//               scanned into start rows (the presum of Section 3.2), and every
//               output row finds its run by binary search.  Each tile writes
//               exactly tile_rows rows, so long and short runs balance.
// Every check of the stream that fails sets a bit in the launch's error word
// and the tile writes in-bounds placeholder values; nothing traps.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "zf_internal.h"

namespace zfd {

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

// Copy `nbytes` from a 16-byte aligned global address into shared memory,
// 16 bytes per thread per step, and zero 32 bytes after them.
__device__ __forceinline__ void stage(uint32_t* sm, const uint8_t* src, uint32_t nbytes) {
    uint32_t nvec = (nbytes + 15) >> 4;
    uint4* s4 = reinterpret_cast<uint4*>(sm);
    for (uint32_t i = threadIdx.x; i < nvec; i += blockDim.x) s4[i] = ldg16(src + 16ull * i);
    if (threadIdx.x < 2) s4[nvec + threadIdx.x] = make_uint4(0, 0, 0, 0);
}

// Store N consecutive values of type T with the widest aligned vector stores
// (the values are packed into 32-bit words in registers first).
template <class T, int N>
__device__ __forceinline__ void store_vec(T* dst, const T (&v)[N]) {
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

// CTA-wide exclusive scan of one uint64 per thread.  `scratch` holds 33 words.
__device__ __forceinline__ uint64_t cta_exclusive_scan(uint64_t v, uint64_t* scratch, uint64_t* total) {
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    uint64_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint64_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
        if (lane >= (uint32_t)d) x += y;
    }
    if (lane == 31) scratch[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t s = lane < nwarps ? scratch[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            uint64_t y = __shfl_up_sync(0xFFFFFFFFu, s, d);
            if (lane >= (uint32_t)d) s += y;
        }
        scratch[lane] = s;  // inclusive prefix of warp sums
    }
    __syncthreads();
    uint64_t warp_pre = warp ? scratch[warp - 1] : 0;
    if (total) *total = scratch[nwarps - 1];
    return warp_pre + x - v;
}

// ---------------------------------------------------------------- Fully-Parallel
// SCHEME: ZF_FOR_BP, ZF_DICT_BP or ZF_RAW.  Rows [r0, r0+nr) of the chunk.
template <class T, int SCHEME>
__device__ void fp_tile(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* sm, uint32_t* err) {
    constexpr int V = 16 / sizeof(T);
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    if constexpr (SCHEME == ZF_RAW) {
        const T* src = reinterpret_cast<const T*>(c.blob + h.off[0]) + r0;
        for (uint32_t g = threadIdx.x; g * V < nr; g += blockDim.x) {
            uint32_t i0 = g * V;
            if (i0 + V <= nr) {
                reinterpret_cast<uint4*>(dst + i0)[0] = ldg16(src + i0);
            } else {
                for (uint32_t i = i0; i < nr; i++) dst[i] = src[i];
            }
        }
        return;
    } else {
    const uint32_t b = h.b;
    const uint8_t* sec = c.blob + h.off[SCHEME == ZF_DICT_BP ? 1 : 0];
    if (b > 8 * sizeof(T) || (SCHEME == ZF_DICT_BP && b > 16)) {
        if (threadIdx.x == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    stage(sm, sec + ((uint64_t)r0 * b >> 3), (uint32_t)(((uint64_t)nr * b + 7) >> 3));
    __syncthreads();
    const T* dict = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const T ref = (T)h.ref;
    bool bad = false;
    for (uint32_t g = threadIdx.x; g * V < nr; g += blockDim.x) {
        uint32_t i0 = g * V;
        T v[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            uint64_t u = extract(sm, (i0 + k) * b, b);
            if (SCHEME == ZF_FOR_BP) {
                v[k] = (T)(ref + (T)u);
            } else {
                bad |= u >= h.n_aux;
                v[k] = u < h.n_aux ? __ldg(dict + u) : (T)0;
            }
        }
        if (i0 + V <= nr) store_vec<T, V>(dst + i0, v);
        else
            for (uint32_t i = i0; i < nr; i++) dst[i] = v[i - i0];
    }
    if (bad) report(err, ZF_ECORRUPT, c.chunk_id);
    __syncthreads();
    }
}

// ---------------------------------------------------------------- delta (Group-Parallel)
// x_j = base + j*min_d + sum_{k=1..j} u_k within each 1024-row block.
template <class T, int VT>
__device__ void delta_tile(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* sm,
                           uint64_t* scan, uint32_t* err) {
    using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
    const uint8_t* table = c.blob + h.off[0];
    const uint8_t* payload = c.blob + h.off[1];
    const uint32_t width = 8 * sizeof(T);
    for (uint32_t blk = r0 / zf::kDeltaBlock; blk * zf::kDeltaBlock < r0 + nr; blk++) {
        const uint8_t* e = table + (uint64_t)blk * zf::kDeltaEntry;
        // 24-byte entry: base, min_d, payload offset, b (8-byte aligned)
        uint2 e0 = __ldg(reinterpret_cast<const uint2*>(e));
        uint2 e1 = __ldg(reinterpret_cast<const uint2*>(e + 8));
        uint2 e2 = __ldg(reinterpret_cast<const uint2*>(e + 16));
        uint64_t base = ((uint64_t)e0.y << 32) | e0.x;
        uint64_t min_d = ((uint64_t)e1.y << 32) | e1.x;
        uint32_t poff = e2.x, b = e2.y & 0xFF;
        uint32_t row0 = blk * zf::kDeltaBlock;
        uint32_t mk = min(zf::kDeltaBlock, h.rows - row0);
        uint32_t nbytes = (mk * b + 7) >> 3;
        bool ok = b <= width && (poff & 15) == 0 && (uint64_t)poff + nbytes <= h.len[1];
        if (!ok) {
            if (threadIdx.x == 0) report(err, ZF_ECORRUPT, c.chunk_id);
            continue;
        }
        stage(sm, payload + poff, nbytes);
        __syncthreads();
        const uint32_t j0 = threadIdx.x * VT;
        U u[VT];
        U local = 0;
#pragma unroll
        for (int k = 0; k < VT; k++) {
            uint32_t j = j0 + k;
            U x = (j < mk && j > 0) ? (U)extract(sm, j * b, b) : (U)0;
            local += x;
            u[k] = local;
        }
        uint64_t pre = cta_exclusive_scan((uint64_t)local, scan, nullptr);
        T out[VT];
#pragma unroll
        for (int k = 0; k < VT; k++) {
            uint32_t j = j0 + k;
            out[k] = (T)(U)((U)base + (U)j * (U)min_d + (U)pre + u[k]);
        }
        T* dst = reinterpret_cast<T*>(c.dst) + row0 + j0;
        if (j0 + VT <= mk) store_vec<T, VT>(dst, out);
        else
            for (uint32_t k = 0; j0 + k < mk; k++) dst[k] = out[k];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- RLE (Group-Parallel)
// Shared memory: starts[cap] (int32) then values[cap] (T).
template <class T>
__device__ void rle_tile(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nr, uint32_t* sm,
                         uint64_t* scan, uint32_t cap, uint32_t* err) {
    constexpr int V = 16 / sizeof(T);
    const T* vals = reinterpret_cast<const T*>(c.blob + h.off[0]);
    const uint32_t* lens = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const uint2* dir = reinterpret_cast<const uint2*>(c.blob + h.off[2]);
    const uint32_t R = h.n_aux;
    uint2 e0 = __ldg(dir + r0 / zf::kRleDirRows);
    uint32_t rf = e0.x, skip = e0.y, rl;
    uint32_t next_skip = 0;
    bool last_tile = r0 + nr >= h.rows;
    bool bad = false;
    if (!last_tile) {
        uint2 e1 = __ldg(dir + (r0 + nr) / zf::kRleDirRows);
        next_skip = e1.y;
        if (e1.y == 0 && e1.x == 0) bad = true;
        rl = e1.y > 0 ? e1.x : e1.x - 1;
    } else {
        rl = R - 1;
    }
    if (r0 == 0 && (rf != 0 || skip != 0)) bad = true;
    if (bad || R == 0 || rf > rl || rl >= R || rl - rf + 1 > cap) {
        if (threadIdx.x == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t m = rl - rf + 1;
    int32_t* starts = reinterpret_cast<int32_t*>(sm);
    T* rv = reinterpret_cast<T*>(sm + ((cap + 3) & ~3u));
    // Load the tile's runs; each thread takes a contiguous slice for the scan.
    const uint32_t per = (m + blockDim.x - 1) / blockDim.x;
    const uint32_t lo = min(m, threadIdx.x * per), hi = min(m, lo + per);
    uint64_t local = 0;
    for (uint32_t i = lo; i < hi; i++) {
        uint32_t L = __ldg(lens + rf + i);
        bad |= L == 0;
        starts[i] = (int32_t)L;
        local += L;
    }
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) rv[i] = __ldg(vals + rf + i);
    uint64_t total;
    uint64_t pre = cta_exclusive_scan(local, scan, &total);
    // presum: start row of each run relative to the tile (the first run may start before it)
    int64_t run = (int64_t)pre - (int64_t)skip;
    for (uint32_t i = lo; i < hi; i++) {
        int32_t L = starts[i];
        starts[i] = (int32_t)run;
        run += L;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // The tile's runs must cover exactly [0, nr): the first run starts at or
        // before row 0 and the last run ends at nr (or continues into the next tile
        // by the amount the next directory entry says).
        int64_t end = (int64_t)total - (int64_t)skip;
        bool ok = skip < (m > 1 ? (uint32_t)(starts[1] + (int32_t)skip) : (uint32_t)total);
        if (last_tile || next_skip == 0) ok &= end == (int64_t)nr;
        else ok &= (int64_t)starts[m - 1] + next_skip == (int64_t)nr && end > (int64_t)nr;
        if (!ok) report(err, ZF_ECORRUPT, c.chunk_id);
    }
    if (bad) report(err, ZF_ECORRUPT, c.chunk_id);
    T* dst = reinterpret_cast<T*>(c.dst) + r0;
    for (uint32_t g = threadIdx.x; g * V < nr; g += blockDim.x) {
        uint32_t i0 = g * V;
        // last run whose start is <= i0
        uint32_t a = 0, z = m;
        while (z - a > 1) {
            uint32_t mid = (a + z) >> 1;
            if (starts[mid] <= (int32_t)i0) a = mid;
            else z = mid;
        }
        T v[V];
#pragma unroll
        for (int k = 0; k < V; k++) {
            while (a + 1 < m && starts[a + 1] <= (int32_t)(i0 + k)) a++;
            v[k] = rv[a];
        }
        if (i0 + V <= nr) store_vec<T, V>(dst + i0, v);
        else
            for (uint32_t i = i0; i < nr; i++) dst[i] = v[i - i0];
    }
    __syncthreads();
}

}  // namespace zfd
