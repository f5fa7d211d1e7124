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
// stream's bytes [a0, a1) of s2 come through a 64-bit buffer, next byte in
// the top bits.  Per row: the slot entry of x mod M gives the value and
// x = f (x >> 12) + (slot - c); then zero, one or two bytes enter while
// x < L (after a step x >= 2^11): one funnel shift of x over the buffer's
// top word, and the buffer moves up by as many bytes.  A row takes at most
// two bytes, so the buffer is topped up to 64 bits before every four rows,
// by every lane at once (no lane waits on another's refill): two aligned
// 8-byte loads from the word holding the next byte (words past the stream's
// last one read as zero; s2 starts on a 16-byte boundary of the blob, so a
// word holding a stream byte lies inside the blob).  Bytes past the stream
// may enter the buffer; a valid stream never takes them.
// Eight int32 or four int64 rows leave as one 32-byte sector.  Returns true
// if the stream is malformed: it must use exactly its bytes and end at x = L.
// SMALL (a chunk of at most four values): the symbol of a slot is found by
// comparing it with the cumulative frequencies, held in registers with the
// frequencies and values, so a row's dependent chain has no shared-memory
// lookup (whose address is the previous row's state).
template <class T, bool SMALL>
__device__ __forceinline__ bool ans_stream(const AnsSmem& sm, const uint8_t* s2, uint32_t a0, uint32_t a1, T* dst,
                                           uint32_t n) {
    const unsigned long long* w8 = reinterpret_cast<const unsigned long long*>(s2);
    const uint32_t lastw = (a1 - 1) >> 3;   // the last word holding a stream byte (a1 > a0)
    uint32_t pos = a0;                      // next stream byte to enter the buffer
    unsigned long long bb = 0;              // buffered bytes, the next one in bits 63..56
    uint32_t nbits = 0;                     // buffered bits, a multiple of 8 in [0, 64]
    auto topup = [&]() {
        const uint32_t need = (64u - nbits) >> 3;
        const uint32_t wi = pos >> 3, s = 8u * (pos & 7u);
        const unsigned long long w0 = wi <= lastw ? __ldg(w8 + wi) : 0ull;
        const unsigned long long w1 = wi + 1 <= lastw ? __ldg(w8 + wi + 1) : 0ull;
        // the 8 bytes from pos, little-endian: (w1:w0) >> s
        const bool lo = s < 32;
        const uint32_t q0 = lo ? (uint32_t)w0 : (uint32_t)(w0 >> 32), q1 = lo ? (uint32_t)(w0 >> 32) : (uint32_t)w1,
                       q2 = lo ? (uint32_t)w1 : (uint32_t)(w1 >> 32);
        const uint32_t r0 = __funnelshift_r(q0, q1, s & 31u), r1 = __funnelshift_r(q1, q2, s & 31u);
        // in stream order from the top, the first `need` of them
        unsigned long long r = ((unsigned long long)__byte_perm(r0, 0, 0x0123) << 32) | __byte_perm(r1, 0, 0x0123);
        r = need ? r & (~0ull << (64u - 8u * need)) : 0ull;
        bb |= nbits < 64 ? r >> nbits : 0ull;
        nbits += 8u * need;
        pos += need;
    };
    topup();
    // the state: bytes a0 .. a0 + 3, little-endian
    uint32_t x = __byte_perm((uint32_t)(bb >> 32), 0, 0x0123);
    bb <<= 32;
    nbits -= 32;
    const uint32_t* val32 = reinterpret_cast<const uint32_t*>(sm.val);
    // SMALL: cumulative frequencies c1..c3 (M past the last symbol), frequencies and values
    uint32_t c1 = 0, c2 = 0, c3 = 0, f0 = 0, f1 = 0, f2 = 0, f3 = 0;
    T v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if constexpr (SMALL) {
        c1 = sm.cum[1];
        c2 = c1 < zf::kAnsM ? sm.cum[2] : zf::kAnsM;
        c3 = c2 < zf::kAnsM ? sm.cum[3] : zf::kAnsM;
        const uint32_t c4 = c3 < zf::kAnsM ? sm.cum[4] : zf::kAnsM;
        f0 = c1;
        f1 = c2 - c1;
        f2 = c3 - c2;
        f3 = c4 - c3;
        v0 = (T)sm.val[0];
        v1 = c1 < zf::kAnsM ? (T)sm.val[1] : v0;
        v2 = c2 < zf::kAnsM ? (T)sm.val[2] : v0;
        v3 = c3 < zf::kAnsM ? (T)sm.val[3] : v0;
    }
    auto step = [&]() -> T {
        T v;
        if constexpr (SMALL) {
            const uint32_t slot = x & (zf::kAnsM - 1u);
            const bool b1 = slot >= c1, b2 = slot >= c2, b3 = slot >= c3;
            const uint32_t c = b3 ? c3 : b2 ? c2 : b1 ? c1 : 0u;
            const uint32_t f = b3 ? f3 : b2 ? f2 : b1 ? f1 : f0;
            v = b3 ? v3 : b2 ? v2 : b1 ? v1 : v0;
            x = f * (x >> zf::kAnsScale) + slot - c;
        } else {
            const uint32_t t = sm.slot[x & (zf::kAnsM - 1u)];
            if constexpr (sizeof(T) == 4) v = (T)val32[2 * (t >> 24)];   // the low word of the 64-bit pattern
            else v = (T)sm.val[t >> 24];
            x = ((t & 0xFFFu) + 1u) * (x >> zf::kAnsScale) + ((t >> 12) & 0xFFFu);
        }
        const uint32_t s = (x < zf::kAnsL ? 8u : 0u) + (x < (zf::kAnsL >> 8) ? 8u : 0u);
        x = __funnelshift_l((uint32_t)(bb >> 32), x, s);
        bb <<= s;
        nbits -= s;
        return v;
    };
    constexpr uint32_t V = 32 / sizeof(T);
    const bool al32 = (reinterpret_cast<uintptr_t>(dst) & 31) == 0;
    uint32_t i0 = 0;
    for (; i0 + V <= n; i0 += V) {
        T v[V];
#pragma unroll
        for (uint32_t e = 0; e < V; e++) {
            if (e % 4 == 0) topup();
            v[e] = step();
        }
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
    }
    for (uint32_t e = 0; i0 < n; i0++, e++) {
        if (e % 4 == 0) topup();
        dst[i0] = step();
    }
    const uint32_t used = (pos - a0) - nbits / 8;   // bytes the rows took
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
    // symbols from the one holding its first slot (binary search on cum);
    // chunks of at most four values decode from the cumulative frequencies
    if (nd > 4) {
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
            bad = nd <= 4 ? ans_stream<int64_t, true>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int64_t*>(c.dst) + r0, n)
                          : ans_stream<int64_t, false>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int64_t*>(c.dst) + r0, n);
        } else {
            bad = nd <= 4 ? ans_stream<int32_t, true>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int32_t*>(c.dst) + r0, n)
                          : ans_stream<int32_t, false>(sm, c.blob + h.off[2], a0, a1, reinterpret_cast<int32_t*>(c.dst) + r0, n);
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
