// zf_plan.cpp -- choice of scheme and chunk size for a column (the Nesting
// Layer's per-column decision of Section 3.2, made here by a size model; the
// learned selector and exhaustive measurement live in zf_select.cpp).
#include <algorithm>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "zf_internal.h"

namespace zf {

// Exact compressed payload size of each integer scheme over chunks of
// `chunk_rows` rows (headers included), from one pass over the data.
template <class T>
void scheme_sizes(const T* x, uint64_t n, uint32_t chunk_rows, uint64_t out[ZF_NSCHEMES]) {
    using U = typename std::make_unsigned<T>::type;
    for (int s = 0; s < ZF_NSCHEMES; s++) out[s] = 0;
    out[ZF_LZ77] = ~0ull;
    out[ZF_FLOAT2INT] = ~0ull;
    out[ZF_STRDICT] = ~0ull;
    out[ZF_ANS] = ~0ull;
    for (uint64_t r0 = 0; r0 < n; r0 += chunk_rows) {
        uint32_t m = (uint32_t)std::min<uint64_t>(chunk_rows, n - r0);
        const T* y = x + r0;
        const uint64_t hdr = kChunkHeader + 16;
        out[ZF_RAW] += hdr + align16((uint64_t)m * sizeof(T));
        T mn = y[0], mx = y[0];
        uint64_t runs = 1;
        for (uint32_t i = 1; i < m; i++) {
            mn = std::min(mn, y[i]);
            mx = std::max(mx, y[i]);
            runs += y[i] != y[i - 1];
        }
        out[ZF_FOR_BP] += hdr + align16(packed_bytes(m, bits_of((uint64_t)(U)((U)mx - (U)mn))));
        out[ZF_RLE] += hdr + align16(runs * sizeof(T)) + align16(runs * 4) + align16(8ull * ((m + 1023) / 1024));
        uint64_t delta = align16(24ull * ((m + 1023) / 1024));
        for (uint32_t b0 = 0; b0 < m; b0 += kDeltaBlock) {
            uint32_t mk = std::min(kDeltaBlock, m - b0);
            T dmin = 0, dmax = 0;
            for (uint32_t j = 1; j < mk; j++) {
                T d = (T)(U)((U)y[b0 + j] - (U)y[b0 + j - 1]);
                if (j == 1 || d < dmin) dmin = d;
                if (j == 1 || d > dmax) dmax = d;
            }
            delta += align16(packed_bytes(mk, bits_of((uint64_t)(U)((U)dmax - (U)dmin))));
        }
        out[ZF_DELTA_BP] += hdr + delta;
        // distinct values, stopping above the dictionary limit
        std::unordered_set<T> seen;
        seen.reserve(1024);
        bool over = false;
        for (uint32_t i = 0; i < m && !over; i++) {
            seen.insert(y[i]);
            over = seen.size() > kMaxDict;
        }
        if (over || out[ZF_DICT_BP] == ~0ull) {
            out[ZF_DICT_BP] = ~0ull;
        } else {
            uint64_t nd = seen.size();
            out[ZF_DICT_BP] += hdr + align16(nd * sizeof(T)) + align16(packed_bytes(m, nd ? bits_of(nd - 1) : 0));
        }
    }
}

template void scheme_sizes<int32_t>(const int32_t*, uint64_t, uint32_t, uint64_t*);
template void scheme_sizes<int64_t>(const int64_t*, uint64_t, uint32_t, uint64_t*);

// Heuristic choice: the scheme with the fewest compressed bytes; ties go to
// the scheme with the cheaper decode (earlier in the enum).
int heuristic_scheme(const zf_column& col, uint32_t chunk_rows) {
    if (col.dtype == ZF_BYTES) return ZF_LZ77;
    if (col.dtype == ZF_F64) return ZF_FLOAT2INT;   // the one float scheme; non-decimals become exceptions
    uint64_t sz[ZF_NSCHEMES];
    if (col.dtype == ZF_I32) scheme_sizes((const int32_t*)col.data, col.n, chunk_rows, sz);
    else scheme_sizes((const int64_t*)col.data, col.n, chunk_rows, sz);
    int best = ZF_RAW;
    for (int s = ZF_FOR_BP; s <= ZF_RLE; s++)
        if (sz[s] < sz[best]) best = s;
    return best;
}

}  // namespace zf

// ---------------------------------------------------------------- Johnson's rule
// Section 3.3 orders the chunks of a call for the two-stage flow (host-to-
// device copy, then decode) with Johnson's rule (S. M. Johnson, "Optimal two-
// and three-stage production schedules with setup times included", 1954):
// the jobs whose copy is shorter than their decode come first, by increasing
// copy time, then the others, by decreasing decode time.  The order minimizes
// the makespan of the two-machine flow shop.  Ties keep the input order.
namespace zf {
void johnson_sequence(const double* copy, const double* dec, uint32_t n, uint32_t* order) {
    for (uint32_t i = 0; i < n; i++) order[i] = i;
    std::stable_sort(order, order + n, [&](uint32_t x, uint32_t y) {
        const bool fx = copy[x] < dec[x], fy = copy[y] < dec[y];
        if (fx != fy) return fx;
        return fx ? copy[x] < copy[y] : dec[x] > dec[y];
    });
}
}  // namespace zf

extern "C" zf_status zf_johnson_order(const float* copy_ms, const float* decode_ms, uint32_t n, uint32_t* order) {
    if (n && (!copy_ms || !decode_ms || !order)) return ZF_EINVAL;
    std::vector<double> c(copy_ms, copy_ms + n), d(decode_ms, decode_ms + n);
    for (uint32_t i = 0; i < n; i++)
        if (!(c[i] >= 0) || !(d[i] >= 0)) return ZF_EINVAL;   // negative or NaN
    zf::johnson_sequence(c.data(), d.data(), n, order);
    return ZF_OK;
}
