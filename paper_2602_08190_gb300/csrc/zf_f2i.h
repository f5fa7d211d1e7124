// zf_f2i.h -- the value of a Float2Int integer with integer instructions only.
//
// Float2Int (Section 2.1, paired with bit-packing in Table 2) stores a double
// v as an integer d with v = d / 10^e for a decimal exponent e of its chunk;
// the decoded value is the double nearest to d / 10^e (|d| <= 2^53, e <= 18).
// A GB300 SM issues few FP64 instructions per clock, so a decoder built on
// the FP64 pipe (a multiply and two fused multiply-adds per value) stays far
// below memory bandwidth.  This file computes the same double with integer
// multiplies, after the Eisel-Lemire idea (D. Lemire, "Number Parsing at a
// Gigabyte per Second", Software: Practice and Experience, 2021): multiply
// the normalized significand by a truncated power of five and fall back to a
// wider product only when the rounding is not yet decided.
//
// d / 10^e = (d / 5^e) * 2^-e; the power of two only moves the exponent, so
// the work is the correctly rounded quotient a / 5^e, a = |d|.  With A = a
// shifted left until bit 63 is set (lz places) and R = ceil(2^(64+s)/5^e),
// s = floor(log2 5^e), the top word H of A * R is the quotient scaled by
// 2^(64+s+lz-64), within the error bounds below:
//   - the product is at or above the exact quotient (R is rounded up) by less
//     than 2^-9 of the result's half-ulp, and dropping the low word of the
//     product costs at most 2^-9 of it more, the other way;
//   - a / 5^e is never exactly halfway between two doubles: a halfway point
//     is a dyadic rational, while a / 5^e (not an integer unless 5^e divides
//     a, and then a double exactly) has the factor 5^e in its denominator.
//     Its distance from any halfway point is at least 1 / 5^e > 2^-42 of the
//     half-ulp (the numerator of the difference is a non-zero integer).
// So H's round bit decides the rounding unless the nine bits below it are all
// zeros (just above a halfway point) or all ones under a zero round bit (just
// below one): then the 128-bit reciprocal R128 = ceil(2^(128+s)/5^e) brings
// the error under 2^-73 of the half-ulp, far inside the 2^-42 gap, and its
// round bit decides.  Neither path needs the bits below the round bit for
// ties, because no ties occur.
#pragma once
#include <stdint.h>

#include "zf_f2i_table.h"

#if defined(__CUDACC__)
#define ZF_F2I_HD __host__ __device__ __forceinline__
#else
#define ZF_F2I_HD inline
#endif

namespace zf {

// One row of the reciprocal table (see gen_f2i_table.py).
struct F2IRecip {
    uint64_t r64, r128_hi, r128_lo;
    uint32_t s;
};

constexpr int64_t kF2IDMax = (int64_t)1 << 53;   // |d| of a valid stream is at most 2^53

ZF_F2I_HD uint64_t f2i_mulhi(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

ZF_F2I_HD int f2i_clz(uint64_t a) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

// The 64-bit pattern of the double nearest d / 10^e, for |d| <= 2^53 and
// 0 <= e <= 18 (`r` = row e of the table; unused when e = 0).  The result is
// assembled as m + ((E + 1022) << 52) from the 53-bit significand m (leading
// one included) and the unbiased exponent E: when rounding carries m to
// 2^53, the sum moves into the next binade by itself.
ZF_F2I_HD uint64_t f2i_bits(int64_t d, uint32_t e, const F2IRecip& r) {
    const uint64_t sign = d < 0 ? (1ull << 63) : 0ull;
    const uint64_t a = d < 0 ? 0ull - (uint64_t)d : (uint64_t)d;
    if (a == 0) return 0;   // +0.0 (a negative zero is always an exception)
    const int lz = f2i_clz(a);
    const uint64_t A = a << lz;
    if (e == 0)             // the integer itself: exact, its top 53 bits are all of it
        return sign | ((A >> 11) + ((uint64_t)(1022 + 63 - lz) << 52));
    uint64_t H = f2i_mulhi(A, r.r64);
    uint32_t ub = (uint32_t)(H >> 63);   // H is in [2^62, 2^64)
    // round bit and the nine bits below it (all in the low word): undecided at 0x1FF and 0x200
    if (((((uint32_t)H >> ub) & 0x3FFu) - 0x1FFu) < 2u) {
        // bits 128..191 of A * R128 (exact, carry included)
        const uint64_t p1h = f2i_mulhi(A, r.r128_hi), p1l = A * r.r128_hi;
        const uint64_t p2h = f2i_mulhi(A, r.r128_lo);
        const uint64_t lo = p1l + p2h;
        H = p1h + (lo < p1l ? 1ull : 0ull);
        ub = (uint32_t)(H >> 63);
    }
    // round to nearest on the round bit (bit 9 + ub): ((H >> (9 + ub)) + 1) >> 1, from H >> 1 so the add cannot wrap
    const uint64_t m = ((H >> 1) + (1ull << (8 + ub))) >> (9 + ub);
    const int E = 62 + (int)ub - lz - (int)r.s - (int)e;
    return sign | (m + ((uint64_t)(E + 1022) << 52));
}

// The same double for a chunk whose integers all lie in [0, 2^32), e >= 1:
// with a < 2^32 the normalized A = A32 * 2^32 (A32 = a shifted until bit 31
// is set), so the top word of A * R is A32 * R_hi + mulhi32(A32, R_lo), one
// wide multiply-add, and every shift is a 32-bit one.  `kexp` is the chunk's
// 1052 - s - e: the biased exponent of the result is kexp + ub - clz32(a).
// Equal to f2i_bits(a, e, r) for every such a (the rare undecided rounding
// takes the general path).
ZF_F2I_HD uint64_t f2i_bits_u32(uint32_t a, uint32_t e, const F2IRecip& r, int32_t kexp) {
#if defined(__CUDA_ARCH__)
    const int lz = __clz((int)a);                 // 32 for a = 0 (the result is then replaced by +0.0)
#else
    const int lz = a ? __builtin_clz(a) : 32;
#endif
    const uint32_t A32 = a << (lz & 31);
#if defined(__CUDA_ARCH__)
    const uint32_t hi32 = __umulhi(A32, (uint32_t)r.r64);
#else
    const uint32_t hi32 = (uint32_t)(((uint64_t)A32 * (uint32_t)r.r64) >> 32);
#endif
    const uint64_t H = (uint64_t)A32 * (r.r64 >> 32) + hi32;
    const uint32_t ub = (uint32_t)(H >> 63);
    const uint32_t t = (uint32_t)H >> ub;
    if (((t & 0x3FFu) - 0x1FFu) < 2u) return a ? f2i_bits((int64_t)a, e, r) : 0ull;
    // m = H >> (10 + ub) rounded on bit 9 + ub (t's bit 9)
    const uint32_t sh = 10u + ub;
    const uint32_t hi = (uint32_t)(H >> 32), lo = (uint32_t)H;
#if defined(__CUDA_ARCH__)
    const uint32_t mlo = __funnelshift_r(lo, hi, sh);
#else
    const uint32_t mlo = (lo >> sh) | (hi << (32 - sh));
#endif
    const uint64_t m = (((uint64_t)(hi >> sh) << 32) | mlo) + ((t >> 9) & 1u);
    const uint64_t bits = m + ((uint64_t)(uint32_t)(kexp + (int)ub - lz) << 52);
    return a ? bits : 0ull;
}

}  // namespace zf
