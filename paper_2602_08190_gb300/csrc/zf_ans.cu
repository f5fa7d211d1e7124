// zf_ans.cu -- dictionary + range ANS decode.  Section 2.1 lists ANS among
// the entropy-based algorithms and Section 3.1 takes its decode as the
// Non-Parallel example: each decode state follows from the one before, so
// the parallelism comes from decoding many independent streams at once.  A
// chunk's rows are cut into streams of 2^k rows (header byte 48; the chunk
// size Section 5.2.3 varies); one warp job takes up to 32 streams of one
// chunk, one per lane, and the four warps of a CTA take consecutive jobs of
// the same chunk (every chunk's jobs are padded to a multiple of four).  The
// rANS coder is Duda's range variant with byte-wise renormalization; the
// layout is described with the container format in zf.h.
#include <cuda_runtime.h>

#include "zf_device.cuh"
#include "zf_launch.h"

namespace {

constexpr uint32_t kWarps = zf::kAnsJobsPerCta;   // warps (jobs) per CTA, all of one chunk

// The CTA's tables for its chunk.  Slot entry: symbol << 24 | (slot - c) <<
// 12 | (f - 1), so a decode step finds the symbol, its frequency f and the
// slot's offset in the symbol's range [c, c + f) with one shared load.
struct AnsSmem {
    uint32_t slot[zf::kAnsM];
    unsigned long long val[zf::kAnsMaxSymbols];   // the symbols' values (64-bit patterns)
    uint32_t cum[zf::kAnsMaxSymbols + 1];         // cumulative frequencies, cum[nd] = M
    uint32_t wsum[kWarps];
};

// Stream k of the chunk, rows [k L, k L + n), decoded by one lane.  The
// stream's bytes [a0, a1) of s2 come through a 64-bit buffer refilled with
// aligned 8-byte loads (s2 starts on a 16-byte boundary of the blob, so a
// word holding a byte of the stream lies inside the blob).  Per row: the
// slot entry of x mod M gives the value and x = f (x >> 12) + (slot - c);
// then zero, one or two bytes enter while x < L (after a step x >= 2^11).
// One refill per row keeps enough bytes buffered: a refill runs when 0 or 8
// bits are left and adds at least one byte, and 0 bits are left only after
// a row that took two bytes from 16 -- which leaves x >= 2^27, so the next
// step gives x >= 2^15 and takes at most one byte.
// Eight int32 or four int64 rows leave as one 32-byte sector.  Returns true
// if the stream is malformed: it must use exactly its bytes and end at x = L.
template <class T>
__device__ __forceinline__ bool ans_stream(const AnsSmem& sm, const uint8_t* s2, uint32_t a0, uint32_t a1, T* dst,
                                           uint32_t n) {
    const unsigned long long* w8 = reinterpret_cast<const unsigned long long*>(s2);
    uint32_t pos = a0;                 // next stream byte to enter the buffer
    unsigned long long bb = 0;         // buffered bytes, the next one lowest
    uint32_t nbits = 0;                // buffered bits (a multiple of 8, <= 64)
    auto refill = [&]() {
        if (pos < a1) {
            const unsigned long long w = __ldg(w8 + (pos >> 3));
            const uint32_t sh = pos & 7u, avail = min(8u - sh, (64u - nbits) >> 3);
            const unsigned long long got = avail == 8 ? w : (w >> (8 * sh)) & ((1ull << (8 * avail)) - 1);
            bb |= got << nbits;
            nbits += 8 * avail;
            pos += avail;
        }
    };
    refill();
    if (nbits < 32) refill();
    uint32_t x = (uint32_t)bb;         // the state: bytes a0 .. a0 + 3, little-endian
    bb >>= 32;
    nbits -= 32;
    uint32_t used = 4;                 // stream bytes consumed
    constexpr uint32_t V = 32 / sizeof(T);
    const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    for (uint32_t i0 = 0; i0 < n; i0 += V) {
        T v[V];
#pragma unroll
        for (uint32_t e = 0; e < V; e++) {
            v[e] = T(0);
            if (i0 + e < n) {
                if (nbits < 16) refill();
                const uint32_t t = sm.slot[x & (zf::kAnsM - 1u)];
                v[e] = (T)sm.val[t >> 24];
                x = ((t & 0xFFFu) + 1u) * (x >> zf::kAnsScale) + ((t >> 12) & 0xFFFu);
                const uint32_t k = (x < zf::kAnsL ? 1u : 0u) + (x < (zf::kAnsL >> 8) ? 1u : 0u);
                const uint32_t lo = (uint32_t)bb;
                x = k == 2 ? (x << 16) | __byte_perm(lo, 0, 0x4401) : k == 1 ? (x << 8) | (lo & 0xFFu) : x;
                bb >>= 8 * k;
                nbits = nbits >= 8 * k ? nbits - 8 * k : 0u;
                used += k;
            }
        }
        if (i0 + V <= n) {
            if (al32) {
                if constexpr (sizeof(T) == 4)
                    zfd::store32(dst + i0, ((unsigned long long)(uint32_t)v[1] << 32) | (uint32_t)v[0],
                                 ((unsigned long long)(uint32_t)v[3] << 32) | (uint32_t)v[2],
                                 ((unsigned long long)(uint32_t)v[5] << 32) | (uint32_t)v[4],
                                 ((unsigned long long)(uint32_t)v[7] << 32) | (uint32_t)v[6]);
                else
                    zfd::store32(dst + i0, (uint64_t)v[0], (uint64_t)v[1], (uint64_t)v[2], (uint64_t)v[3]);
            } else {
                zfd::store_vec<T, V>(dst + i0, v);
            }
        } else {
#pragma unroll
            for (uint32_t e = 0; e < V; e++)
                if (i0 + e < n) dst[i0 + e] = v[e];
        }
    }
    return used != a1 - a0 || x != zf::kAnsL;
}

// The CTA builds its chunk's tables, then warp w decodes job blockIdx.x *
// kWarps + w: lane i takes the job's stream i.
__global__ void __launch_bounds__(kWarps * 32) ans_kernel(const ZfDevChunk* chunks, uint32_t nchunks, uint32_t njobs,
                                                           uint32_t* err) {
    __shared__ AnsSmem sm;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t job0 = blockIdx.x * kWarps;
    if (job0 >= njobs) return;
    uint32_t a = 0, z = nchunks;
    while (z - a > 1) {
        const uint32_t mid = (a + z) >> 1;
        if (__ldg(&chunks[mid].tile0) <= job0) a = mid;
        else z = mid;
    }
    const ZfDevChunk c = chunks[a];
    zfd::Hdr h;
    zfd::load_hdr(c.blob, h);
    const uint32_t sz = c.dtype == ZF_I64 ? 8u : 4u;
    const uint32_t lg = c.blob[48], nd = h.n_aux;
    const uint32_t L = 1u << (lg & 31u);
    const uint32_t K = (lg >= zf::kAnsLogMin && lg <= zf::kAnsLogMax) ? (h.rows + L - 1) / L : 0u;
    const uint32_t fb = (2u * nd + 3u) & ~3u;
    // header and section bounds (checked on the host too; the device does not rely on it)
    bool ok = h.rows == c.rows && (uint64_t)c.rows * sz <= c.dst_cap && (c.dtype == ZF_I32 || c.dtype == ZF_I64) &&
              h.b == zf::kAnsScale && nd > 0 && nd <= zf::kAnsMaxSymbols && K > 0 && h.ref == K &&
              h.len[0] == nd * sz && h.len[1] == fb + 4u * (K + 1u);
    for (int s = 0; s < 3; s++)
        ok = ok && h.off[s] >= 64 && !(h.off[s] & 15) && (uint64_t)h.off[s] + h.len[s] <= c.blob_bytes;
    if (!ok) {
        if (tid == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;   // uniform over the CTA
    }
    // frequencies, two per thread, and their exclusive scan over the CTA
    const uint16_t* fq = reinterpret_cast<const uint16_t*>(c.blob + h.off[1]);
    const uint32_t i0 = 2 * tid;
    const uint32_t f0 = i0 < nd ? (uint32_t)__ldg(fq + i0) : 0u, f1 = i0 + 1 < nd ? (uint32_t)__ldg(fq + i0 + 1) : 0u;
    const bool fbad = (i0 < nd && f0 == 0) || (i0 + 1 < nd && f1 == 0);
    const uint32_t pair = f0 + f1;
    const uint32_t incl = zfd::warp_incl_sum<uint32_t>(pair, lane);
    if (lane == 31) sm.wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (uint32_t q = 0; q < kWarps; q++) {
        before += q < warp ? sm.wsum[q] : 0u;
        total += sm.wsum[q];
    }
    if (__syncthreads_or(fbad) || total != zf::kAnsM) {
        if (tid == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t c0 = before + incl - pair;
    if (i0 < nd) sm.cum[i0] = c0;
    if (i0 + 1 < nd) sm.cum[i0 + 1] = c0 + f0;
    if (tid == 0) sm.cum[nd] = zf::kAnsM;
    for (uint32_t k = tid; k < nd; k += kWarps * 32)
        sm.val[k] = sz == 8 ? (unsigned long long)__ldg(reinterpret_cast<const int64_t*>(c.blob + h.off[0]) + k)
                            : (unsigned long long)(uint32_t)__ldg(reinterpret_cast<const int32_t*>(c.blob + h.off[0]) + k);
    __syncthreads();
    // slot entries: thread t fills slots [t * 32, t * 32 + 32), walking the
    // symbols from the one holding its first slot (binary search on cum)
    {
        constexpr uint32_t per = zf::kAnsM / (kWarps * 32);
        const uint32_t first = tid * per;
        uint32_t lo = 0, hi = nd - 1;   // the last symbol whose cum is <= first
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (sm.cum[mid] <= first) lo = mid;
            else hi = mid - 1;
        }
        uint32_t s = lo, cs = sm.cum[s], ce = sm.cum[s + 1];
        for (uint32_t slot = first; slot < first + per; slot++) {
            while (slot >= ce) {
                s++;
                cs = ce;
                ce = sm.cum[s + 1];
            }
            sm.slot[slot] = (s << 24) | ((slot - cs) << 12) | (ce - cs - 1u);
        }
    }
    __syncthreads();
    // one stream per lane
    const uint32_t job = job0 + warp;
    const uint32_t k = (job - c.tile0) * zf::kAnsStreamsPerJob + lane;
    bool bad = false;
    if (k < K) {
        const uint32_t* starts = reinterpret_cast<const uint32_t*>(c.blob + h.off[1] + fb);
        const uint32_t a0 = __ldg(starts + k), a1 = __ldg(starts + k + 1);
        const uint32_t r0 = k * L, n = min(L, h.rows - r0);
        if (a1 < a0 || a1 - a0 < 4u || a1 > h.len[2]) {
            bad = true;
        } else if (sz == 8) {
            bad = ans_stream<int64_t>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int64_t*>(c.dst) + r0, n);
        } else {
            bad = ans_stream<int32_t>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int32_t*>(c.dst) + r0, n);
        }
    }
    if (bad) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
}

}  // namespace

namespace zf {

// njobs is a multiple of kAnsJobsPerCta: every chunk's jobs are padded to it.
cudaError_t launch_ans(const ZfDevChunk* chunks, uint32_t nchunks, uint32_t njobs, uint32_t* err, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    ans_kernel<<<(njobs + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(chunks, nchunks, njobs, err);
    return cudaGetLastError();
}

}  // namespace zf
