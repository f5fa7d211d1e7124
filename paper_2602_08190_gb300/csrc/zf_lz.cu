// zf_lz.cu -- LZ77 decode, the Non-Parallel pattern of Section 3.1: blocks
// of 64 KiB decode independently, each by one warp.  (Section 4 schedules one
// thread per chunk; here the 32 lanes of a warp share one block, 32 tokens
// at a time.)  Section 2.1 names LZ77; the block layout is this library's,
// described with the format in zf.h.
#include <cuda_runtime.h>

#include "zf_device.cuh"
#include "zf_launch.h"

namespace {

// One warp decodes one block, 32 tokens at a time (lane i holds token t0+i).
//   Lengths: the LEB128 lengths stream is read 32 bytes per step, one byte per
//   lane; a ballot of the bytes without a continuation bit locates the ends
//   of the varints, each end lane assembles its value from the bytes of the
//   lanes before it (shuffles), and the values go to a ring in shared memory.
//   Positions: two warp scans of the lengths give every token of the batch
//   its literal range in s2 and its output range, so the whole batch is
//   validated before a byte moves.
//   Window (a batch whose output fits kLzWin): the batch is assembled in a
//   shared-memory window placed at the output's alignment mod 16, then written
//   out with 16-byte stores.  Literals: the batch's literal bytes are
//   contiguous in s2; the lanes copy them 32 at a time, each finding its token
//   by a binary search over the lanes' literal starts.  Matches: byte k of a
//   match at p with offset `off` equals out[p + k - off].  Every lane first
//   copies, from global memory, the bytes of its match whose source precedes
//   the batch (final already); then the matches whose sources reach into the
//   batch are finished in token order inside the window: the bytes k < off
//   from before p, then the bytes k >= off as out[p + (k mod off)], so a match
//   that overlaps its own output repeats its source.
//   Direct (any other batch): output goes straight to global memory in
//   rounds.  Every output byte before the first unfinished match is final, so
//   every match whose source ends there is ready; the ready matches' bytes are
//   copied as one flat list (all loads of a group issued before its stores),
//   and the round repeats.  The first unfinished match is always ready.
constexpr uint32_t kLzLenRing = 512;   // pre-parsed lengths per warp
constexpr uint32_t kLzBatch = 480;     // lengths parsed ahead per refill (at most ring - 32)
constexpr uint32_t kLzWin = 4096;      // batch output window per warp
constexpr uint32_t kFull = 0xFFFFFFFFu;

struct LzParse {
    uint32_t vp = 0;        // next byte of the lengths stream
    uint32_t parsed = 0;    // lengths parsed so far
    uint32_t carry = 0;     // value bits of a varint cut by the last step
    uint32_t carry_n = 0;   // its bytes so far
    bool bad = false;
};

// One 32-byte step of the lengths stream; `byte` is this lane's byte (0x80
// past the end).
__device__ __forceinline__ void lz_parse_step(uint32_t byte, uint32_t l0, uint32_t* lr, LzParse& ps, uint32_t lane) {
    const bool valid = ps.vp + lane < l0;
    const uint32_t ends = __ballot_sync(kFull, valid && !(byte & 0x80u));
    const uint32_t b1 = __shfl_up_sync(kFull, byte, 1);
    const uint32_t b2 = __shfl_up_sync(kFull, byte, 2);
    bool bad = false;
    if ((ends >> lane) & 1) {
        const uint32_t below = ends & ((1u << lane) - 1u);
        const int pt = below ? 31 - __clz(below) : -1;   // previous end in this step
        const uint32_t n = lane - pt;                    // bytes of this varint in this step
        uint32_t v = byte & 0x7Fu, nb = n;
        if (n >= 2) v = (b1 & 0x7Fu) | (v << 7);
        if (n >= 3) v = (b2 & 0x7Fu) | (v << 7);
        if (pt < 0 && ps.carry_n) {                      // continues the varint cut by the last step
            v = ps.carry | (v << (7 * ps.carry_n));
            nb += ps.carry_n;
        }
        bad = nb > 3;
        lr[(ps.parsed + __popc(below)) & (kLzLenRing - 1)] = v;
    }
    // bytes after the last end start a varint that the next step finishes
    const int last = ends ? 31 - __clz(ends) : -1;
    uint32_t tail = min(32u, l0 - ps.vp) - (uint32_t)(last + 1);
    uint32_t tv = 0;
    for (uint32_t j = 0; j < tail && j < 3; j++)
        tv |= (__shfl_sync(kFull, byte, last + 1 + j) & 0x7Fu) << (7 * j);
    if (last < 0) {                                      // the whole step continued the varint
        tv = ps.carry | (tv << (7 * ps.carry_n));
        tail += ps.carry_n;
    }
    ps.carry = tv;
    ps.carry_n = tail;
    ps.parsed += __popc(ends);
    ps.vp += 32;
    ps.bad = __any_sync(kFull, bad || tail > 3) || ps.bad;
}

// Parse lengths until `upto` are available (or the stream ends); the bytes of
// eight steps are loaded before the first is used.
__device__ __forceinline__ void lz_parse(const uint8_t* s0, uint32_t l0, uint32_t* lr, LzParse& ps, uint32_t upto,
                                         uint32_t lane) {
    while (!ps.bad && ps.parsed < upto && ps.vp < l0) {
        uint32_t by[8];
#pragma unroll
        for (uint32_t q = 0; q < 8; q++) {
            const uint32_t pos = ps.vp + 32 * q + lane;
            by[q] = pos < l0 ? __ldg(s0 + pos) : 0x80u;
        }
#pragma unroll
        for (uint32_t q = 0; q < 8; q++) {
            if (ps.bad || ps.parsed >= upto || ps.vp >= l0) break;
            lz_parse_step(by[q], l0, lr, ps, lane);
        }
    }
    if (ps.vp > l0) ps.vp = l0;
    __syncwarp();
}

// Largest lane i whose `start` (nondecreasing over the lanes) is <= j.
__device__ __forceinline__ uint32_t lz_find(uint32_t start, uint32_t j) {
    uint32_t i = 0;
#pragma unroll
    for (uint32_t s = 16; s; s >>= 1)
        if (__shfl_sync(kFull, start, i + s) <= j) i += s;
    return i;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ void lz_block(const ZfDevChunk& c, uint32_t* lr, uint8_t* win, uint32_t* err) {
    const uint32_t lane = threadIdx.x & 31;
    zfd::Hdr h;
    zfd::load_hdr(c.blob, h);
    uint8_t* dst = c.dst;
    if (h.rows != c.rows || h.rows > zf::kLzBlock || h.rows > c.dst_cap) {
        if (lane == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    const uint8_t* s0 = c.blob + h.off[0];
    if (h.flags & 1) {  // stored raw
        uint32_t n16 = h.rows >> 4;
        for (uint32_t i = lane; i < n16; i += 32)
            reinterpret_cast<uint4*>(dst)[i] = zfd::ldg16(s0 + 16 * i);
        for (uint32_t i = n16 * 16 + lane; i < h.rows; i += 32) dst[i] = s0[i];
        return;
    }
    const uint16_t* offs = reinterpret_cast<const uint16_t*>(c.blob + h.off[1]);
    const uint8_t* lit = c.blob + h.off[2];
    const uint32_t T = h.n_aux, l0 = h.len[0], l2 = h.len[2], rows = h.rows;
    const uint32_t nlen = 2 * T - 1;                         // lengths in the stream
    bool ok = T > 0 && h.len[1] == 2 * (T - 1);
    if (!ok) {
        if (lane == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
        return;
    }
    // the three streams are read once, front to back: start them towards L2
    for (uint32_t i = 128 * lane; i < l0; i += 4096) prefetch_l2(s0 + i);
    for (uint32_t i = 128 * lane; i < h.len[1]; i += 4096) prefetch_l2(c.blob + h.off[1] + i);
    for (uint32_t i = 128 * lane; i < l2; i += 4096) prefetch_l2(lit + i);
    LzParse ps;
    uint32_t lp = 0, op = 0;                                 // literal and output bytes done
    uint32_t off_next = lane + 1 < T ? __ldg(offs + lane) : 0;  // offsets are loaded one batch ahead
    for (uint32_t t0 = 0; t0 < T; t0 += 32) {
        const uint32_t nt = min(32u, T - t0);
        const uint32_t need = min(nlen, 2 * (t0 + nt));      // the last token has no match length
        if (ps.parsed < need) {
            lz_parse(s0, l0, lr, ps, min(nlen, 2 * t0 + kLzBatch), lane);
            if (ps.bad || ps.parsed < need) { ok = false; break; }
        }
        const uint32_t t = t0 + lane;
        const bool has_m = lane < nt && t + 1 < T;
        const uint32_t ll = lane < nt ? lr[(2 * t) & (kLzLenRing - 1)] : 0;
        const uint32_t ml = has_m ? lr[(2 * t + 1) & (kLzLenRing - 1)] + zf::kLzMinMatch : 0;
        const uint32_t off = has_m ? off_next : 0;
        off_next = t + 33 < T ? __ldg(offs + t + 32) : 0;
        uint32_t lend = ll, oend = ll + ml;                  // inclusive sums over the lanes
#pragma unroll
        for (uint32_t d = 1; d < 32; d <<= 1) {
            const uint32_t a = __shfl_up_sync(kFull, lend, d), b = __shfl_up_sync(kFull, oend, d);
            if (lane >= d) { lend += a; oend += b; }
        }
        lend += lp;
        oend += op;
        const uint32_t lstart = lend - ll, mpos = oend - ml, ostart = mpos - ll;
        // lengths are below 2^21, so none of the sums wrap
        const bool bad = lend > l2 || oend > rows || (has_m && (off == 0 || off > mpos));
        if (__any_sync(kFull, bad)) { ok = false; break; }
        const uint32_t lb = __shfl_sync(kFull, lend, 31) - lp;
        const uint32_t src = mpos - off;
        const uint32_t ob = __shfl_sync(kFull, oend, 31) - op;
        if (ob + 16 <= kLzWin) {
            // window byte x holds output byte op + x - a; base + x is its global address
            const uint32_t a = (uint32_t)(reinterpret_cast<uintptr_t>(dst + op) & 15);
            uint8_t* base = dst + op - a;
            // the bytes of each match whose source precedes the batch: aligned
            // words over [src, src + g) -- the last ends before op + 3, inside
            // the block, because this match still has ml >= 4 bytes from
            // mpos >= op.  The first four words are loaded here, so that their
            // latency overlaps the literals' loads.
            const uint32_t d = a + mpos - op;
            const uint32_t g = (has_m && src < op) ? min(min(ml, off), op - src) : 0;
            const uint32_t sh = src & 3u, nw = g ? (sh + g + 3) >> 2 : 0;
            const uint32_t* ws = reinterpret_cast<const uint32_t*>(dst + (src - sh));
            uint32_t x[4];
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) x[q] = q < nw ? ws[q] : 0;
            for (uint32_t bl = 0; bl < lb; bl += 128) {
                uint32_t v[4];
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t jj = bl + 32 * q + lane;
                    v[q] = jj < lb ? __ldg(lit + lp + jj) : 0;
                }
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    if (bl + 32 * q >= lb) break;
                    const uint32_t j = lp + bl + 32 * q + lane;
                    const uint32_t i = lz_find(lstart, j);
                    const uint32_t os = __shfl_sync(kFull, ostart, i), ls = __shfl_sync(kFull, lstart, i);
                    if (j < lp + lb) win[a + os - op + (j - ls)] = (uint8_t)v[q];
                }
            }
            for (uint32_t w0 = 0; w0 < nw; w0 += 4) {
                if (w0) {
#pragma unroll
                    for (uint32_t q = 0; q < 4; q++) x[q] = w0 + q < nw ? ws[w0 + q] : 0;
                }
#pragma unroll
                for (uint32_t q = 0; q < 4; q++)
#pragma unroll
                    for (uint32_t b = 0; b < 4; b++) {
                        const uint32_t kb = 4 * (w0 + q) + b;
                        if (kb >= sh && kb < sh + g) win[d + kb - sh] = (uint8_t)(x[q] >> (8 * b));
                    }
            }
            __syncwarp();
            // the rest, in token order, inside the window
            uint32_t todo = __ballot_sync(kFull, has_m && g < ml);
            while (todo) {
                const uint32_t i = __ffs(todo) - 1;
                todo &= todo - 1;
                const uint32_t di = __shfl_sync(kFull, d, i), mi = __shfl_sync(kFull, ml, i);
                const uint32_t oi = __shfl_sync(kFull, off, i), gi = __shfl_sync(kFull, g, i);
                const uint32_t c1 = min(mi, oi);
                for (uint32_t k = gi + lane; k < c1; k += 32) win[di + k] = win[di + k - oi];
                __syncwarp();
                if (oi < mi) {
                    for (uint32_t k = oi + lane; k < mi; k += 32) win[di + k] = win[di + k % oi];
                    __syncwarp();
                }
            }
            // write the window out: head bytes, 16-byte words, tail bytes
            const uint32_t e = a + ob, x0 = (a + 15) & ~15u, x1 = e & ~15u;
            if (x0 <= x1) {
                if (lane < x0 - a) base[a + lane] = win[a + lane];
                for (uint32_t w = (x0 >> 4) + lane; w < (x1 >> 4); w += 32)
                    reinterpret_cast<uint4*>(base)[w] = reinterpret_cast<const uint4*>(win)[w];
                if (lane < e - x1) base[x1 + lane] = win[x1 + lane];
            } else {
                if (lane < ob) base[a + lane] = win[a + lane];
            }
            __syncwarp();
            lp = __shfl_sync(kFull, lend, 31);
            op = __shfl_sync(kFull, oend, 31);
            continue;
        }
        // direct: literals
        for (uint32_t base = 0; base < lb; base += 128) {
            uint32_t v[4];
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                const uint32_t jj = base + 32 * q + lane;
                v[q] = jj < lb ? __ldg(lit + lp + jj) : 0;
            }
#pragma unroll
            for (uint32_t q = 0; q < 4; q++) {
                if (base + 32 * q >= lb) break;
                const uint32_t j = lp + base + 32 * q + lane;
                const uint32_t i = lz_find(lstart, j);
                const uint32_t os = __shfl_sync(kFull, ostart, i), ls = __shfl_sync(kFull, lstart, i);
                if (j < lp + lb) dst[os + (j - ls)] = (uint8_t)v[q];
            }
        }
        __syncwarp();
        // matches, in rounds
        uint32_t pend = __ballot_sync(kFull, has_m);
        while (pend) {
            const uint32_t hwm = __shfl_sync(kFull, mpos, __ffs(pend) - 1);
            const bool ready = ((pend >> lane) & 1) && src + min(ml, off) <= hwm;
            const uint32_t len = ready ? ml : 0;
            uint32_t cend = len;
#pragma unroll
            for (uint32_t d = 1; d < 32; d <<= 1) {
                const uint32_t a = __shfl_up_sync(kFull, cend, d);
                if (lane >= d) cend += a;
            }
            const uint32_t total = __shfl_sync(kFull, cend, 31), cstart = cend - len;
            for (uint32_t base = 0; base < total; base += 128) {
                uint32_t v[4], to[4];
#pragma unroll
                for (uint32_t q = 0; q < 4; q++) {
                    const uint32_t jj = base + 32 * q + lane;
                    const uint32_t i = lz_find(cstart, jj);
                    const uint32_t k = jj - __shfl_sync(kFull, cstart, i);
                    const uint32_t o = __shfl_sync(kFull, off, i), m = __shfl_sync(kFull, ml, i);
                    const uint32_t s = __shfl_sync(kFull, src, i) + (o >= m ? k : k % o);
                    to[q] = __shfl_sync(kFull, mpos, i) + k;
                    v[q] = jj < total ? dst[s] : 0;
                }
#pragma unroll
                for (uint32_t q = 0; q < 4; q++)
                    if (base + 32 * q + lane < total) dst[to[q]] = (uint8_t)v[q];
            }
            __syncwarp();
            pend &= ~__ballot_sync(kFull, ready);
        }
        lp = __shfl_sync(kFull, lend, 31);
        op = __shfl_sync(kFull, oend, 31);
    }
    // every length used, no varint left open, every literal and output byte accounted for
    if (ok) ok = !ps.bad && ps.parsed == nlen && ps.carry_n == 0 && ps.vp >= l0 && op == rows && lp == l2;
    if (!ok && lane == 0) zfd::report(err, ZF_ECORRUPT, c.chunk_id);
}

__global__ void __launch_bounds__(32, 32) lz_kernel(const ZfDevChunk* chunks, uint32_t n, uint32_t* err) {
    __shared__ uint32_t lens[kLzLenRing];
    __shared__ __align__(16) uint8_t win[kLzWin];
    for (uint32_t k = blockIdx.x; k < n; k += gridDim.x) {
        const ZfDevChunk c = chunks[k];
        lz_block(c, lens, win, err);
        __syncwarp();
    }
}

}  // namespace

namespace zf {

cudaError_t launch_lz(const ZfDevChunk* chunks, uint32_t n, uint32_t* err, int num_sms, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    // one warp (one block) per CTA, so a small launch still spreads over
    // every SM; up to 32 CTAs per SM, then warps loop over the rest
    uint32_t blocks = n;
    uint32_t cap = (uint32_t)num_sms * 32;
    if (blocks > cap) blocks = cap;
    lz_kernel<<<blocks, 32, 0, s>>>(chunks, n, err);
    return cudaGetLastError();
}

}  // namespace zf
