// zf_ans.cu -- dictionary + range ANS decode.  Section 2.1 lists ANS among
// the entropy-based algorithms and Section 3.1 takes its decode as the
// Non-Parallel example: each decode state follows from the one before, so
// the parallelism comes from decoding many independent streams at once.  A
// chunk's rows are cut into 512-row streams; one warp job takes up to 32
// streams of one chunk, one per lane.  The rANS coder is Duda's range
// variant with byte-wise renormalization; the layout is described with the
// container format in zf.h.
#include <cuda_runtime.h>

#include "zf_device.cuh"
#include "zf_launch.h"

namespace {

constexpr uint32_t kWarps = 4;   // warps (jobs) per CTA

// A warp's tables for one chunk.
struct AnsSmem {
    uint8_t sym[zf::kAnsM];        // symbol of every slot x mod M
    uint32_t fc[256];              // frequency | cumulative frequency << 16
    unsigned long long val[256];   // the symbols' values (64-bit patterns)
};

// Streams [k0, k0 + 32) of a chunk.  The warp first builds the slot table:
// lane l loads the frequencies of symbols 8l..8l+7, one warp scan gives the
// cumulative frequencies, and lane l fills slots [128 l, 128 l + 128) by
// walking the symbols from the one holding its first slot.  Then lane l
// decodes stream k0 + l alone: per row the symbol of slot x mod M, its value,
// x = f * (x / M) + slot - c, and up to two bytes while x < L; four (int32)
// or two (int64) rows leave in one 16-byte store.  Frequencies that do not
// fill M, streams that run out of bytes or do not end at x = L, and stream
// bounds outside s2 are reported.
template <class T>
__device__ void ans_streams(const ZfDevChunk& c, const zfd::Hdr& h, uint32_t k0, AnsSmem& sm, uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nd = h.n_aux, rows = h.rows;
    const uint32_t K = (rows + zf::kAnsStream - 1) / zf::kAnsStream;
    const uint32_t fb = (2u * nd + 3u) & ~3u;
    if (h.b != zf::kAnsScale || nd == 0 || nd > zf::kAnsMaxSymbols || h.ref != K ||
        h.len[0] != nd * (uint32_t)sizeof(T) || h.len[1] != fb + 4u * (K + 1u) || k0 >= K) {
        if (lane == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    // ---- tables
    const uint16_t* fq = reinterpret_cast<const uint16_t*>(c.blob + h.off[1]);
    const T* vals = reinterpret_cast<const T*>(c.blob + h.off[0]);
    uint32_t f[8], sum = 0;
    bool bad = false;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const uint32_t k = 8 * lane + e;
        f[e] = k < nd ? (uint32_t)__ldg(fq + k) : 0u;
        bad |= k < nd && f[e] == 0;
        sum += f[e];
    }
    const uint32_t incl = zfd::warp_incl_sum<uint32_t>(sum, lane);
    bad |= __shfl_sync(0xFFFFFFFFu, incl, 31) != zf::kAnsM;
    if (__any_sync(0xFFFFFFFFu, bad)) {
        if (lane == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    uint32_t cum = incl - sum;
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const uint32_t k = 8 * lane + e;
        if (k < nd) sm.fc[k] = f[e] | (cum << 16);
        cum += f[e];
    }
    for (uint32_t k = lane; k < nd; k += 32) sm.val[k] = (unsigned long long)__ldg(vals + k);
    __syncwarp();
    {
        const uint32_t first = 128u * lane;
        uint32_t lo = 0, hi = nd - 1;   // the last symbol whose cumulative frequency is <= first
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if ((sm.fc[mid] >> 16) <= first) lo = mid;
            else hi = mid - 1;
        }
        uint32_t s = lo, fcs = sm.fc[s];
        for (uint32_t slot = first; slot < first + 128u; slot++) {
            while (slot >= (fcs >> 16) + (fcs & 0xFFFFu) && s + 1 < nd) fcs = sm.fc[++s];
            sm.sym[slot] = (uint8_t)s;
        }
    }
    __syncwarp();
    // ---- one stream per lane
    const uint32_t k = k0 + lane;
    if (k < K) {
        const uint32_t* starts = reinterpret_cast<const uint32_t*>(c.blob + h.off[1] + fb);
        const uint8_t* s2 = c.blob + h.off[2];
        const uint32_t a0 = __ldg(starts + k), a1 = __ldg(starts + k + 1);
        const uint32_t r0 = k * zf::kAnsStream, n = min(zf::kAnsStream, rows - r0);
        bool sbad = a1 < a0 || a1 - a0 < 4u || a1 > h.len[2];
        if (!sbad) {
            uint32_t x = (uint32_t)s2[a0] | ((uint32_t)s2[a0 + 1] << 8) | ((uint32_t)s2[a0 + 2] << 16) |
                         ((uint32_t)s2[a0 + 3] << 24);
            uint32_t p = a0 + 4;
            T* dst = reinterpret_cast<T*>(c.dst) + r0;
            constexpr uint32_t V = 16 / sizeof(T);
            for (uint32_t i0 = 0; i0 < n && !sbad; i0 += V) {
                T v[V];
#pragma unroll
                for (uint32_t e = 0; e < V; e++) {
                    v[e] = T(0);
                    if (i0 + e < n && !sbad) {
                        const uint32_t slot = x & (zf::kAnsM - 1u);
                        const uint32_t s = sm.sym[slot], fcs = sm.fc[s];
                        v[e] = (T)sm.val[s];
                        x = (fcs & 0xFFFFu) * (x >> zf::kAnsScale) + slot - (fcs >> 16);
                        // after a step x >= 2^11, so two bytes bring it back to [L, 256 L)
#pragma unroll
                        for (int r = 0; r < 2; r++) {
                            if (x < zf::kAnsL) {
                                if (p < a1) x = (x << 8) | s2[p++];
                                else sbad = true;
                            }
                        }
                        sbad |= x < zf::kAnsL;
                    }
                }
                if (i0 + V <= n) {
                    uint32_t w[4];
                    memcpy(w, v, 16);   // register moves: the store needs no aligned local copy
                    reinterpret_cast<uint4*>(dst + i0)[0] = make_uint4(w[0], w[1], w[2], w[3]);
                } else {
#pragma unroll
                    for (uint32_t e = 0; e < V; e++)
                        if (i0 + e < n) dst[i0 + e] = v[e];
                }
            }
            sbad |= x != zf::kAnsL || p != a1;
        }
        if (sbad) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
    }
}

// One warp job per warp: job j of a chunk covers its streams [32 j, 32 j + 32).
__global__ void __launch_bounds__(kWarps * 32) ans_kernel(const ZfDevChunk* chunks, uint32_t nchunks,
                                                           uint32_t njobs, uint32_t* err) {
    __shared__ AnsSmem sm[kWarps];
    const uint32_t warp = threadIdx.x >> 5;
    const uint32_t job = blockIdx.x * kWarps + warp;
    if (job >= njobs) return;
    uint32_t a = 0, z = nchunks;
    while (z - a > 1) {
        const uint32_t mid = (a + z) >> 1;
        if (__ldg(&chunks[mid].tile0) <= job) a = mid;
        else z = mid;
    }
    const ZfDevChunk c = chunks[a];
    zfd::Hdr h;
    zfd::load_hdr(c.blob, h);
    const uint32_t sz = c.dtype == ZF_I64 ? 8u : 4u;
    if (h.rows != c.rows || (uint64_t)c.rows * sz > c.dst_cap || (c.dtype != ZF_I32 && c.dtype != ZF_I64)) {
        if ((threadIdx.x & 31) == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t k0 = (job - c.tile0) * zf::kAnsStreamsPerJob;
    if (c.dtype == ZF_I64) ans_streams<int64_t>(c, h, k0, sm[warp], err);
    else ans_streams<int32_t>(c, h, k0, sm[warp], err);
}

}  // namespace

namespace zf {

cudaError_t launch_ans(const ZfDevChunk* chunks, uint32_t nchunks, uint32_t njobs, uint32_t* err, cudaStream_t s) {
    if (njobs == 0) return cudaSuccess;
    ans_kernel<<<(njobs + kWarps - 1) / kWarps, kWarps * 32, 0, s>>>(chunks, nchunks, njobs, err);
    return cudaGetLastError();
}

}  // namespace zf
