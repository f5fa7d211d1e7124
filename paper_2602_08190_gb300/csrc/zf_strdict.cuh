// zf_strdict.cuh -- the string-dictionary decoder (Group-Parallel pattern):
// a byte column stored as bit-packed codes into a dictionary of tokens
// (Section 2.1 dictionary encoding over the words of a text column, as
// Section 5.3.1 does for the comment column).
#pragma once
#include "zf_device.cuh"

namespace zfd {

// ---------------------------------------------------------------- string dictionary (Group-Parallel)
// A string-dictionary chunk is the dictionary entries of its tokens, one
// after another: token t lands at the sum of the lengths before it (a
// prefix scan, the Group-Parallel pattern).  The encoder stores the output
// offset of every 1024th token, so each 1024-token tile starts on its own.

// Tokens [r0, r0 + nrows) of the chunk (r0 a multiple of 1024; the chunk may
// end sooner).  Per tile the codes are staged in shared memory; 32 tokens at
// a time, lane i takes token t0 + i: its entry's offset and length from the
// dictionary offsets, one warp scan places the 32 entries, each lane copies
// its entry (at most 64 bytes) into a shared-memory window placed at the
// output's alignment mod 16, and the warp writes the window out with 16-byte
// stores.  Codes past the dictionary, entries that leave the dictionary and
// tiles whose lengths do not reach the next tile's start are reported.
__device__ inline void strdict_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                            uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nd = h.n_aux, b = h.b;
    const uint64_t T = h.ref;
    if (nd == 0 || nd > zf::kStrDictMax || b > 16 || T > h.rows || r0 >= T ||
        (uint64_t)h.len[0] < 4ull * (nd + 1 + (T + zf::kStrTile - 1) / zf::kStrTile)) {
        if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t ntok = (uint32_t)min((unsigned long long)nrows, (unsigned long long)(T - r0));
    const uint32_t ntiles = (uint32_t)((T + zf::kStrTile - 1) / zf::kStrTile);
    const uint32_t* doff = reinterpret_cast<const uint32_t*>(c.blob + h.off[0]);
    const uint32_t* tstart = doff + nd + 1;
    const uint8_t* dict = c.blob + h.off[1];
    const uint8_t* codes = c.blob + h.off[2];
    const uint32_t dlen = h.len[1];
    uint32_t* cbuf = wsm;
    uint8_t* win = reinterpret_cast<uint8_t*>(wsm) + kStrCodeBuf;
    bool bad = false;
    for (uint32_t i0 = 0; i0 < ntok && !bad; i0 += zf::kStrTile) {
        const uint32_t tile = (r0 + i0) / zf::kStrTile;
        const uint32_t nt = min(zf::kStrTile, ntok - i0);
        // a tile's codes start at bit tile * 1024 * b: a 16-byte boundary of the section
        stage_async(cbuf, codes + (uint64_t)tile * 128u * b, (nt * b + 7) >> 3, lane);
        __pipeline_commit();
        const uint32_t o0 = __ldg(tstart + tile);
        const uint32_t o1 = tile + 1 < ntiles ? __ldg(tstart + tile + 1) : h.rows;
        bad = o0 > o1 || o1 > h.rows;
        __pipeline_wait_prior(0);
        __syncwarp();
        uint32_t op = o0;
        for (uint32_t t = 0; t < nt && !bad; t += 32) {
            const uint32_t k = t + lane;
            uint32_t a0 = 0, len = 0;
            bool lbad = false;
            if (k < nt) {
                const uint32_t code = b ? (uint32_t)extract(cbuf, k * b, b) : 0u;
                if (code < nd) {
                    a0 = __ldg(doff + code);
                    len = __ldg(doff + code + 1) - a0;
                }
                lbad = code >= nd || len == 0 || len > zf::kStrTokenMax || a0 > dlen || len > dlen - a0;
                if (lbad) len = 0;
            }
            const uint32_t incl = warp_incl_sum<uint32_t>(len, lane);
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31), start = incl - len;
            if (__any_sync(0xFFFFFFFFu, lbad) || total > o1 - op) {
                bad = true;
                break;
            }
            // window byte x holds output byte op + x - a
            const uint32_t a = (uint32_t)(reinterpret_cast<uintptr_t>(c.dst + op) & 15);
            uint8_t* base = c.dst + op - a;
            for (uint32_t q = 0; q < len; q++) win[a + start + q] = __ldg(dict + a0 + q);
            __syncwarp();
            const uint32_t e = a + total, x0 = (a + 15) & ~15u, x1 = e & ~15u;
            if (x0 <= x1) {
                if (lane < x0 - a) base[a + lane] = win[a + lane];
                for (uint32_t w = (x0 >> 4) + lane; w < (x1 >> 4); w += 32)
                    reinterpret_cast<uint4*>(base)[w] = reinterpret_cast<const uint4*>(win)[w];
                if (lane < e - x1) base[x1 + lane] = win[x1 + lane];
            } else if (lane < total) {
                base[a + lane] = win[a + lane];
            }
            __syncwarp();
            op += total;
        }
        bad = bad || op != o1;
    }
    if (bad && lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
}

}  // namespace zfd
