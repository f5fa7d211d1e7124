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

// OR one dictionary entry (`len` bytes at byte `a0` of the dictionary
// section, whose 32-bit words are `dw`, the last one holding entry bytes
// `last_w`) into byte `w0` of a zeroed shared-memory window of 32-bit words.
// Destination word j holds source bytes a0 - (w0 mod 4) + 4j .. + 3: one
// funnel shift of two consecutive source words, read as whole words, four
// destination words per step.  Source words before the entry start are
// inside the chunk (the section starts at byte 64 or later).  Words past the
// section's end only feed bytes the masks drop: with SAFE the chunk holds at
// least 32 bytes after the section (every word read ends within 20 bytes of
// it) and they are read as they are, otherwise they are clamped to the last
// word.  Every word is merged with an atomic OR, so entries that share a
// word need no ordering.
template <bool SAFE>
__device__ __forceinline__ void strdict_copy(uint32_t* win, const uint32_t* dw, int last_w, uint32_t a0, uint32_t len,
                                             uint32_t w0) {
    if (len == 0) return;
    const int base = (int)a0 - (int)(w0 & 3u);           // source byte of destination word 0's byte 0 (>= -3)
    const int ws = base >> 2;                              // its word (floor; -1 at the least)
    const uint32_t sh = 8u * ((uint32_t)base & 3u);
    const uint32_t q0 = w0 >> 2, e = w0 + len;
    const uint32_t nw = ((e + 3) >> 2) - q0;               // destination words
    const uint32_t head_mask = 0xFFFFFFFFu << (8u * (w0 & 3u));
    const uint32_t tail_mask = 0xFFFFFFFFu >> (8u * ((4u - (e & 3u)) & 3u));
    for (uint32_t j0 = 0; j0 < nw; j0 += 4) {
        uint32_t s[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int w = ws + (int)j0 + k;
            s[k] = __ldg(dw + (SAFE ? w : min(w, last_w)));
        }
#pragma unroll
        for (uint32_t jj = 0; jj < 4; jj++) {
            const uint32_t j = j0 + jj;
            if (j < nw) {
                uint32_t m = j + 1 == nw ? tail_mask : 0xFFFFFFFFu;
                if (j == 0) m &= head_mask;
                atomicOr(&win[q0 + j], __funnelshift_r(s[jj], s[jj + 1], sh) & m);
            }
        }
    }
}

// Tokens [r0, r0 + ntok) of the chunk (r0 a multiple of 1024).  Per tile the
// codes are staged in shared memory; 64 tokens at a time, lane i takes
// tokens t0 + 2i and t0 + 2i + 1 (both codes from one extraction): their
// entries' offsets and lengths from the dictionary offsets, one warp scan of
// the lanes' two-token sums places the 64 entries, each lane ORs its entries
// into a zeroed shared-memory window (strdict_copy) and the warp writes the
// window's whole 16-byte blocks out, zeroing them as they leave.  The window
// holds 16 tokens of the 64-byte maximum (a batch that needs more goes
// through it in two or four rounds), so it stays small and the SM's L1 keeps
// room for the dictionary.  The next 64 tokens' entries are loaded
// before the current ones are copied.  The window's byte 0 is the output byte
// at a 16-byte boundary, so every store is a 16-byte vector; the last,
// partial block carries over to the next batch.
// Only the job's first block (whose leading bytes belong to the tokens before
// the job) and its last partial block leave as single bytes.  Codes past the
// dictionary, entries that are empty, longer than 64 bytes or leave the
// dictionary, and tiles whose lengths do not reach the next tile's start are
// reported.
template <bool SAFE>
__device__ __forceinline__ void strdict_tokens(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t ntok,
                                               uint32_t* wsm, uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nd = h.n_aux, b = h.b;
    const uint64_t T = h.ref;
    const uint32_t ntiles = (uint32_t)((T + zf::kStrTile - 1) / zf::kStrTile);
    const uint32_t* doff = reinterpret_cast<const uint32_t*>(c.blob + h.off[0]);
    const uint32_t* tstart = doff + nd + 1;
    const uint32_t* dw = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const uint8_t* codes = c.blob + h.off[2];
    const uint32_t dlen = h.len[1];
    const int last_w = (int)((dlen - 1) >> 2);
    const uint32_t cmask = (1u << b) - 1u;                 // b <= 16
    uint32_t* cbuf = wsm;
    uint32_t* win = wsm + kStrCodeBuf / 4;
    const uint8_t* winb = reinterpret_cast<const uint8_t*>(win);
    for (uint32_t w = lane; w < kStrWin / 4; w += 32) win[w] = 0;
    uint32_t op = __ldg(tstart + r0 / zf::kStrTile);      // output byte of the job's first token
    bool bad = op > h.rows;
    uint32_t a = op & 15u;                                 // window byte a holds output byte op
    uint32_t head = a;                                     // leading bytes of block 0 that are not this job's
    uint8_t* base = c.dst + (op - a);                      // output address of window byte 0 (16-byte aligned)
    __syncwarp();
    for (uint32_t i0 = 0; i0 < ntok && !bad; i0 += zf::kStrTile) {
        const uint32_t tile = (r0 + i0) / zf::kStrTile;
        const uint32_t nt = min(zf::kStrTile, ntok - i0);
        // a tile's codes start at bit tile * 1024 * b: a 16-byte boundary of the section
        stage_async(cbuf, codes + (uint64_t)tile * 128u * b, (nt * b + 7) >> 3, lane);
        __pipeline_commit();
        const uint32_t o0 = __ldg(tstart + tile);
        const uint32_t o1 = tile + 1 < ntiles ? __ldg(tstart + tile + 1) : h.rows;
        bad = o0 != op || o0 > o1 || o1 > h.rows;
        __pipeline_wait_prior(0);
        __syncwarp();
        // entries [a0, e0) and [a1, e1) of tokens k and k + 1 of the staged tile
        auto entry2 = [&](uint32_t k, uint32_t& a0, uint32_t& e0, uint32_t& a1, uint32_t& e1, bool& cbad) {
            a0 = e0 = a1 = e1 = 0;
            cbad = false;
            if (k < nt) {
                const uint32_t pair = b ? (uint32_t)extract(cbuf, k * b, 2 * b) : 0u;
                const uint32_t c0 = pair & cmask, c1 = pair >> b;
                const bool two = k + 1 < nt;
                cbad = c0 >= nd || (two && c1 >= nd);
                if (!cbad) {
                    a0 = __ldg(doff + c0);
                    e0 = __ldg(doff + c0 + 1);
                    if (two) {
                        a1 = __ldg(doff + c1);
                        e1 = __ldg(doff + c1 + 1);
                    }
                }
            }
        };
        uint32_t na0, ne0, na1, ne1;
        bool ncbad;
        entry2(2 * lane, na0, ne0, na1, ne1, ncbad);
        for (uint32_t t = 0; t < nt && !bad; t += 64) {
            const uint32_t a0 = na0, a1 = na1, k = t + 2 * lane;
            uint32_t len0 = ne0 - na0, len1 = ne1 - na1;
            // 1 <= len <= 64 and inside the dictionary, for every token of the tile
            const bool lbad = ncbad || (k < nt && (len0 - 1u >= zf::kStrTokenMax || ne0 > dlen)) ||
                              (k + 1 < nt && (len1 - 1u >= zf::kStrTokenMax || ne1 > dlen));
            if (lbad) len0 = len1 = 0;
            entry2(k + 64, na0, ne0, na1, ne1, ncbad);
            const uint32_t s2 = len0 + len1;
            const uint32_t incl = warp_incl_sum<uint32_t>(s2, lane);
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31), start = incl - s2;
            if (__any_sync(0xFFFFFFFFu, lbad) || total > o1 - op) {
                bad = true;
                break;
            }
            // the batch's bytes go through the window in one round, or, when they
            // would not fit, in two or four rounds of consecutive lanes (a round
            // of eight lanes, 16 tokens of at most 64 bytes, always fits)
            const uint32_t half = __shfl_sync(0xFFFFFFFFu, incl, 15);
            const uint32_t R = a + total + 16u <= kStrWin ? 1u
                               : max(half, total - half) + 31u <= kStrWin ? 2u : 4u;
            const uint32_t per = 32u / R;                            // lanes per round
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t l0 = r * per;
                const uint32_t before = l0 ? __shfl_sync(0xFFFFFFFFu, incl, l0 - 1) : 0u;   // batch bytes of earlier rounds
                const uint32_t rtot = __shfl_sync(0xFFFFFFFFu, incl, l0 + per - 1) - before;
                if (lane - l0 < per) {
                    strdict_copy<SAFE>(win, dw, last_w, a0, len0, a + start - before);
                    strdict_copy<SAFE>(win, dw, last_w, a1, len1, a + start - before + len0);
                }
                __syncwarp();
                // whole blocks out (zeroed behind), block 0 keeping its leading bytes that are not this job's
                const uint32_t e = a + rtot, x1 = e & ~15u;
                if (x1) {
                    if (head) {
                        if (lane >= head && lane < 16) base[lane] = winb[lane];
                        __syncwarp();
                        if (lane < 4) win[lane] = 0;
                    }
                    uint4* wv = reinterpret_cast<uint4*>(win);
                    for (uint32_t q = (head ? 1u : 0u) + lane; q < (x1 >> 4); q += 32) {
                        reinterpret_cast<uint4*>(base)[q] = wv[q];
                        wv[q] = make_uint4(0, 0, 0, 0);
                    }
                    head = 0;
                    __syncwarp();
                    // the partial block [x1, e) becomes block 0 (its old place is zeroed)
                    if (x1 < e && lane < 4) {
                        win[lane] = win[(x1 >> 2) + lane];
                        win[(x1 >> 2) + lane] = 0;
                    }
                    __syncwarp();
                }
                base += x1;
                a = e - x1;
            }
            op += total;
        }
        bad = bad || op != o1;
    }
    // the job's last partial block, byte by byte
    if (!bad && lane >= head && lane < a) base[lane] = winb[lane];
    if (bad && lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
}

__device__ inline void strdict_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                                   uint32_t* err) {
    const uint32_t nd = h.n_aux, b = h.b;
    const uint64_t T = h.ref;
    if (nd == 0 || nd > zf::kStrDictMax || b > 16 || T > h.rows || r0 >= T ||
        (uint64_t)h.len[0] < 4ull * (nd + 1 + (T + zf::kStrTile - 1) / zf::kStrTile) || h.len[1] == 0) {
        if ((threadIdx.x & 31) == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t ntok = (uint32_t)min((unsigned long long)nrows, (unsigned long long)(T - r0));
    if ((uint64_t)h.off[1] + h.len[1] + 32u <= c.blob_bytes) strdict_tokens<true>(c, h, r0, ntok, wsm, err);
    else strdict_tokens<false>(c, h, r0, ntok, wsm, err);
}

}  // namespace zfd
