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

// Copy one dictionary entry (`len` bytes at byte `a0` of the dictionary
// section, whose 32-bit words are `dw`, the last readable one `last_w`) to
// byte `w0` of a shared-memory window of 32-bit words.  The entry is read as
// whole words, four destination words per step: destination word j holds
// source bytes a0 - (w0 mod 4) + 4j .. + 3, one funnel shift of two
// consecutive source words.  Words wholly inside the entry are stored; the
// first and last may share bytes with the neighbouring entries and are
// merged with an atomic OR into the (zeroed) window.
__device__ __forceinline__ void strdict_copy(uint32_t* win, const uint32_t* dw, int last_w, uint32_t a0, uint32_t len,
                                             uint32_t w0) {
    if (len == 0) return;
    const int base = (int)a0 - (int)(w0 & 3u);           // source byte of destination word 0's byte 0 (>= -3)
    const int ws = base >> 2;                              // its word (floor)
    const uint32_t sh = 8u * ((uint32_t)base & 3u);
    const uint32_t q0 = w0 >> 2, e = w0 + len;
    const uint32_t nw = ((e + 3) >> 2) - q0;               // destination words
    const uint32_t head_mask = 0xFFFFFFFFu << (8u * (w0 & 3u));
    const uint32_t tail_mask = (e & 3u) ? 0xFFFFFFFFu >> (8u * (4u - (e & 3u))) : 0xFFFFFFFFu;
    for (uint32_t j0 = 0; j0 < nw; j0 += 4) {
        uint32_t s[5];
#pragma unroll
        for (int k = 0; k < 5; k++) {
            const int w = ws + (int)j0 + k;
            s[k] = (w >= 0 && w <= last_w && j0 + k <= nw) ? __ldg(dw + w) : 0u;
        }
#pragma unroll
        for (uint32_t jj = 0; jj < 4; jj++) {
            const uint32_t j = j0 + jj;
            if (j < nw) {
                uint32_t v = __funnelshift_r(s[jj], s[jj + 1], sh);
                uint32_t m = 0xFFFFFFFFu;
                if (j == 0) m &= head_mask;
                if (j + 1 == nw) m &= tail_mask;
                if (m == 0xFFFFFFFFu) win[q0 + j] = v;
                else atomicOr(&win[q0 + j], v & m);
            }
        }
    }
}

// Tokens [r0, r0 + nrows) of the chunk (r0 a multiple of 1024; the chunk may
// end sooner).  32 tokens at a time, lane i takes token t0 + i: its code
// (read straight from the packed stream: the lanes' codes are consecutive
// bits, so the loads coalesce), its entry's offset and length from the
// dictionary offsets -- for the next 32 tokens these loads are issued before
// the current 32 are copied -- one warp scan places the 32 entries, each lane
// copies its entry into a shared-memory window (strdict_copy) and the warp
// writes the window's whole 16-byte blocks out.  A warp holds only its 2 KiB
// window in shared memory, so most of the SM's L1 is left to the
// dictionaries.  The window's byte 0 is the output byte at a 16-byte
// boundary, so every store is a 16-byte vector; the last, partial block
// carries over to the next 32 tokens.  Only the job's first block (whose
// leading bytes belong to the tokens before the job) and its last partial
// block leave as single bytes.  Codes past the dictionary, entries that leave
// the dictionary and tiles whose lengths do not reach the next tile's start
// are reported.
__device__ inline void strdict_job(const ZfDevChunk& c, const Hdr& h, uint32_t r0, uint32_t nrows, uint32_t* wsm,
                                   uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t nd = h.n_aux, b = h.b;
    const uint64_t T = h.ref;
    if (nd == 0 || nd > zf::kStrDictMax || b > 16 || T > h.rows || r0 >= T ||
        (uint64_t)h.len[0] < 4ull * (nd + 1 + (T + zf::kStrTile - 1) / zf::kStrTile) ||
        (uint64_t)h.len[2] < (T * b + 7) / 8) {
        if (lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint32_t ntok = (uint32_t)min((unsigned long long)nrows, (unsigned long long)(T - r0));
    const uint32_t ntiles = (uint32_t)((T + zf::kStrTile - 1) / zf::kStrTile);
    const uint32_t* doff = reinterpret_cast<const uint32_t*>(c.blob + h.off[0]);
    const uint32_t* tstart = doff + nd + 1;
    const uint32_t* dw = reinterpret_cast<const uint32_t*>(c.blob + h.off[1]);
    const uint32_t* cw = reinterpret_cast<const uint32_t*>(c.blob + h.off[2]);
    const uint32_t dlen = h.len[1];
    const int last_w = dlen ? (int)((dlen - 1) >> 2) : -1;
    const uint32_t code_words = (uint32_t)((h.len[2] + 3) >> 2);   // readable words of the packed codes
    uint32_t* win = wsm;
    const uint8_t* winb = reinterpret_cast<const uint8_t*>(win);
    for (uint32_t w = lane; w < kStrWin / 4; w += 32) win[w] = 0;
    uint32_t op = __ldg(tstart + r0 / zf::kStrTile);      // output byte of the job's first token
    bool bad = op > h.rows;
    uint32_t a = op & 15u;                                 // window byte a holds output byte op
    uint32_t head = a;                                     // leading bytes of block 0 that are not this job's
    uint8_t* base = c.dst + (op - a);                      // output address of window byte 0 (16-byte aligned)
    __syncwarp();
    // entry (offset, length) of chunk token k; length 0 and `kb` set if invalid
    auto entry = [&](uint64_t k, bool valid, uint32_t& a0, uint32_t& len, bool& kb) {
        a0 = 0;
        len = 0;
        kb = false;
        if (valid) {
            uint32_t code = 0;
            if (b) {
                const uint64_t bit = k * b;
                const uint32_t wi = (uint32_t)(bit >> 5), sh = (uint32_t)(bit & 31);
                const uint32_t lo = __ldg(cw + wi);
                const uint32_t hi = (sh + b > 32 && wi + 1 < code_words) ? __ldg(cw + wi + 1) : 0u;
                code = __funnelshift_r(lo, hi, sh) & ((1u << b) - 1u);
            }
            if (code < nd) {
                a0 = __ldg(doff + code);
                len = __ldg(doff + code + 1) - a0;
            }
            kb = code >= nd || len == 0 || len > zf::kStrTokenMax || a0 > dlen || len > dlen - a0;
            if (kb) len = 0;
        }
    };
    const uint64_t job0 = r0;
    uint32_t na0, nlen;
    bool nkb;
    entry(job0 + lane, lane < ntok, na0, nlen, nkb);
    for (uint32_t i0 = 0; i0 < ntok && !bad; i0 += zf::kStrTile) {
        const uint32_t tile = (r0 + i0) / zf::kStrTile;
        const uint32_t nt = min(zf::kStrTile, ntok - i0);
        const uint32_t o0 = __ldg(tstart + tile);
        const uint32_t o1 = tile + 1 < ntiles ? __ldg(tstart + tile + 1) : h.rows;
        bad = o0 != op || o0 > o1 || o1 > h.rows;
        for (uint32_t t = 0; t < nt && !bad; t += 32) {
            const uint32_t a0 = na0, len = nlen;
            const bool lbad = nkb;
            const uint32_t incl = warp_incl_sum<uint32_t>(len, lane);
            const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31), start = incl - len;
            if (__any_sync(0xFFFFFFFFu, lbad) || total > o1 - op) {
                bad = true;
                break;
            }
            // the next 32 tokens' entries, loaded while these are copied
            const uint32_t nx = i0 + t + 32 + lane;
            entry(job0 + nx, nx < ntok, na0, nlen, nkb);
            strdict_copy(win, dw, last_w, a0, len, a + start);
            __syncwarp();
            // whole blocks out; block 0 keeps its leading bytes that are not this job's
            const uint32_t e = a + total, x1 = e & ~15u;
            if (x1) {
                if (head) {
                    if (lane >= head && lane < 16) base[lane] = winb[lane];
                }
                for (uint32_t q = (head ? 1u : 0u) + lane; q < (x1 >> 4); q += 32)
                    reinterpret_cast<uint4*>(base)[q] = reinterpret_cast<const uint4*>(win)[q];
                head = 0;
            }
            // the partial block [x1, e) becomes block 0; the rest of the window is zeroed
            const uint32_t tw = lane < 4 ? win[(x1 >> 2) + lane] : 0u;
            __syncwarp();
            for (uint32_t w = lane; w < ((e + 15) >> 4) * 4; w += 32) win[w] = 0;
            __syncwarp();
            if (lane < 4) win[lane] = tw;
            __syncwarp();
            base += x1;
            a = e - x1;
            op += total;
        }
        bad = bad || op != o1;
    }
    // the job's last partial block, byte by byte
    if (!bad && lane >= head && lane < a) base[lane] = winb[lane];
    if (bad && lane == 0) report(err, ZF_ECORRUPT, c.chunk_id);
}

}  // namespace zfd
