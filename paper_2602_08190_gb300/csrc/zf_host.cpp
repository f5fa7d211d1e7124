// zf_host.cpp -- host side of the library: the column encoders that run at
// compression time (Section 3: data is compressed on the CPU and kept in host
// memory), the serializer of the container format, and the structural
// validator used when a serialized column is imported.
//
// Codecs (Section 2.1): FOR + bit-packing, dictionary + bit-packing, delta +
// bit-packing, run-length, LZ77, Float2Int + bit-packing, string dictionary
// + bit-packing, dictionary + ANS.  Encoding is canonical for all but LZ77,
// so two correct encoders produce the same bytes.
#include <cuda_runtime_api.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <functional>
#include <mutex>
#include <string_view>
#include <thread>
#include <unordered_map>

#include "zf_internal.h"

namespace zf {
namespace {

// ---------------------------------------------------------------- byte output
struct Out {
    std::vector<uint8_t> b;
    void put8(uint64_t pos, uint8_t v) { b[pos] = v; }
    void put32(uint64_t pos, uint32_t v) { memcpy(&b[pos], &v, 4); }
    void put64(uint64_t pos, uint64_t v) { memcpy(&b[pos], &v, 8); }
};

// Bit-packing: value i at stream bits [i*b, i*b+b), LSB first.  Writes exactly
// ceil(n*b/8) bytes at `out`.
template <class Get>
void pack_stream(uint64_t n, uint32_t b, Get get, uint8_t* out) {
    if (b == 0) return;
    unsigned __int128 acc = 0;
    uint32_t nacc = 0;
    uint64_t o = 0;
    const uint64_t mask = b >= 64 ? ~0ull : ((1ull << b) - 1);
    for (uint64_t i = 0; i < n; i++) {
        acc |= (unsigned __int128)(get(i) & mask) << nacc;
        nacc += b;
        if (nacc >= 64) {
            uint64_t w = (uint64_t)acc;
            memcpy(out + o, &w, 8);
            o += 8;
            acc >>= 64;
            nacc -= 64;
        }
    }
    uint32_t tail = (nacc + 7) / 8;
    uint64_t w = (uint64_t)acc;
    for (uint32_t k = 0; k < tail; k++) out[o + k] = (uint8_t)(w >> (8 * k));
}

struct ChunkWriter {
    Out& o;
    uint64_t end = kChunkHeader;
    explicit ChunkWriter(Out& out) : o(out) {}
    uint64_t section(int s, uint64_t len) {
        uint64_t off = align16(end);
        o.put32(24 + 4 * s, (uint32_t)off);
        o.put32(36 + 4 * s, (uint32_t)len);
        end = off + len;
        return off;
    }
    void header(int scheme, int dtype, uint32_t bw, uint32_t flags, uint32_t rows, uint32_t n_aux, uint64_t ref) {
        o.put32(0, kChunkMagic);
        o.put8(4, (uint8_t)scheme);
        o.put8(5, (uint8_t)dtype);
        o.put8(6, (uint8_t)bw);
        o.put8(7, (uint8_t)flags);
        o.put32(8, rows);
        o.put32(12, n_aux);
        o.put64(16, ref);
    }
};

template <class T> constexpr int dtype_code() { return sizeof(T) == 8 ? ZF_I64 : ZF_I32; }

// ------------------------------------------------------------------ RAW
template <class T>
void enc_raw(const T* x, uint32_t m, Out& o) {
    o.b.assign(align16(kChunkHeader + (uint64_t)m * sizeof(T)), 0);
    ChunkWriter w(o);
    w.header(ZF_RAW, dtype_code<T>(), 0, 0, m, 0, 0);
    uint64_t off = w.section(0, (uint64_t)m * sizeof(T));
    if (m) memcpy(&o.b[off], x, (uint64_t)m * sizeof(T));
}

// ------------------------------------------------------------------ string dictionary + BP
// Tokens of a byte chunk: cut after each space byte, before each row start,
// after kStrTokenMax bytes and at the chunk end.  The dictionary is the
// distinct tokens in byte order (a prefix first) and each token is stored as
// its rank at bits(ndict - 1) bits (Section 2.1 dictionary encoding over the
// words of a text column, as Section 5.3.1 does for the comment column).
// Above kStrDictMax distinct tokens every byte is a token.  Sections: s0 =
// dictionary offsets [ndict + 1], then the output offset of every
// kStrTile-th token; s1 = the dictionary's bytes; s2 = the codes.
void enc_strdict(const uint8_t* x, uint32_t m, const std::vector<uint8_t>& row_start, Out& o) {
    std::vector<std::pair<uint32_t, uint32_t>> tok;   // (first byte, length)
    std::unordered_map<std::string_view, uint32_t> ids;
    std::vector<std::string_view> dict;
    for (int pass = 0; pass < 2; pass++) {
        tok.clear();
        for (uint32_t i = 0; i < m;) {
            uint32_t j = i + 1;
            if (pass == 0)
                while (j < m && x[j - 1] != ' ' && !row_start[j] && j - i < kStrTokenMax) j++;
            tok.push_back({i, j - i});
            i = j;
        }
        ids.clear();
        dict.clear();
        bool over = false;
        for (auto& t : tok) {
            std::string_view v(reinterpret_cast<const char*>(x) + t.first, t.second);
            if (ids.emplace(v, 0).second) {
                dict.push_back(v);
                if (dict.size() > kStrDictMax) {
                    over = true;
                    break;
                }
            }
        }
        if (!over) break;
    }
    std::sort(dict.begin(), dict.end(), [](std::string_view a, std::string_view b) {
        const size_t n = std::min(a.size(), b.size());
        const int c = n ? memcmp(a.data(), b.data(), n) : 0;
        return c ? c < 0 : a.size() < b.size();
    });
    for (uint32_t k = 0; k < dict.size(); k++) ids[dict[k]] = k;
    const uint32_t nd = (uint32_t)dict.size(), T = (uint32_t)tok.size();
    const uint32_t b = bits_of(nd ? nd - 1 : 0), ntiles = (T + kStrTile - 1) / kStrTile;
    uint64_t dbytes = 0;
    for (auto& v : dict) dbytes += v.size();
    const uint64_t l0 = 4ull * (nd + 1 + ntiles), l2 = packed_bytes(T, b);
    o.b.assign(align16(align16(align16(kChunkHeader + l0) + dbytes) + l2), 0);
    ChunkWriter w(o);
    w.header(ZF_STRDICT, ZF_BYTES, b, 0, m, nd, T);
    const uint64_t s0 = w.section(0, l0), s1 = w.section(1, dbytes);
    uint64_t pos = 0;
    for (uint32_t k = 0; k < nd; k++) {
        o.put32(s0 + 4ull * k, (uint32_t)pos);
        memcpy(&o.b[s1 + pos], dict[k].data(), dict[k].size());
        pos += dict[k].size();
    }
    o.put32(s0 + 4ull * nd, (uint32_t)pos);
    std::vector<uint32_t> code(T);
    uint64_t out = 0;
    for (uint32_t i = 0; i < T; i++) {
        code[i] = ids.find(std::string_view(reinterpret_cast<const char*>(x) + tok[i].first, tok[i].second))->second;
        if (i % kStrTile == 0) o.put32(s0 + 4ull * (nd + 1 + i / kStrTile), (uint32_t)out);
        out += tok[i].second;
    }
    const uint64_t s2 = w.section(2, l2);
    pack_stream(T, b, [&](uint64_t i) { return (uint64_t)code[i]; }, o.b.data() + s2);
}

// ------------------------------------------------------------------ Float2Int + BP
// A double v is stored as the integer d with v = d / 10^e, e the chunk's
// decimal exponent (0..18), and the integers FOR + bit-packed (Section 2.1
// "Float2Int"; Table 2 pairs it with bit-packing).  d decodes to the double
// nearest d / 10^e.  A value that does not come back bit for bit
// from its rounded integer is an exception (row + 64 bits).  The chunk takes
// the exponent with the fewest exceptions, the smallest on a tie.
struct Pow10 {
    double p[kF2IMaxExp + 1];
    Pow10() {
        double x = 1.0;   // exact: 10^18 < 2^63 and every power up to 10^22 is a double
        for (int e = 0; e <= kF2IMaxExp; e++) {
            p[e] = x;
            x *= 10.0;
        }
    }
};
const Pow10 kPow10;

// |d| <= 2^53 and 10^e (e <= 18) are doubles exactly, so one IEEE division
// is the double nearest d / 10^e.
inline double f2i_value(int64_t d, int e) { return (double)d / kPow10.p[e]; }

inline bool f2i_fits(double v, int e, int64_t* d) {
    if (!std::isfinite(v)) return false;
    const double t = v * kPow10.p[e];
    if (!(std::fabs(t) < 9007199254740992.0)) return false;
    const int64_t k = (int64_t)std::nearbyint(t);
    const double back = f2i_value(k, e);
    if (memcmp(&back, &v, 8) != 0) return false;
    *d = k;
    return true;
}

void enc_f2i(const double* x, uint32_t m, Out& o) {
    int best_e = 0;
    uint32_t best_ex = UINT32_MAX;
    for (int e = 0; e <= kF2IMaxExp && best_ex > 0; e++) {
        uint32_t ex = 0;
        int64_t d;
        for (uint32_t i = 0; i < m && ex < best_ex; i++) ex += !f2i_fits(x[i], e, &d);
        if (ex < best_ex) {
            best_ex = ex;
            best_e = e;
        }
    }
    std::vector<int64_t> d(m);
    std::vector<uint8_t> ok(m);
    int64_t mn = 0;
    bool have = false;
    for (uint32_t i = 0; i < m; i++) {
        ok[i] = f2i_fits(x[i], best_e, &d[i]);
        if (ok[i] && (!have || d[i] < mn)) {
            mn = d[i];
            have = true;
        }
    }
    uint64_t mx = 0;
    for (uint32_t i = 0; i < m; i++)
        if (ok[i]) mx = std::max(mx, (uint64_t)d[i] - (uint64_t)mn);
    const uint32_t b = bits_of(mx);
    const uint64_t pb = packed_bytes(m, b);
    o.b.assign(align16(align16(align16(kChunkHeader) + pb) + 4ull * best_ex) + align16(8ull * best_ex) + 16, 0);
    ChunkWriter w(o);
    w.header(ZF_FLOAT2INT, ZF_F64, b, 0, m, best_ex, (uint64_t)mn);
    o.put8(48, (uint8_t)best_e);
    const uint64_t o0 = w.section(0, pb);
    pack_stream(m, b, [&](uint64_t i) { return ok[i] ? (uint64_t)d[i] - (uint64_t)mn : 0ull; }, &o.b[o0]);
    const uint64_t o1 = w.section(1, 4ull * best_ex), o2 = w.section(2, 8ull * best_ex);
    uint32_t k = 0;
    for (uint32_t i = 0; i < m; i++)
        if (!ok[i]) {
            uint64_t bits;
            memcpy(&bits, &x[i], 8);
            memcpy(&o.b[o1 + 4ull * k], &i, 4);
            memcpy(&o.b[o2 + 8ull * k], &bits, 8);
            k++;
        }
    o.b.resize(align16(w.end));
}

// ------------------------------------------------------------------ FOR + BP
template <class T>
void enc_for(const T* x, uint32_t m, Out& o) {
    using U = typename std::make_unsigned<T>::type;
    T mn = m ? x[0] : 0, mx = m ? x[0] : 0;
    for (uint32_t i = 1; i < m; i++) {
        mn = std::min(mn, x[i]);
        mx = std::max(mx, x[i]);
    }
    uint32_t b = bits_of((uint64_t)(U)((U)mx - (U)mn));
    uint64_t pb = packed_bytes(m, b);
    o.b.assign(align16(align16(kChunkHeader) + pb), 0);
    ChunkWriter w(o);
    w.header(ZF_FOR_BP, dtype_code<T>(), b, 0, m, 0, (uint64_t)(int64_t)mn);
    uint64_t off = w.section(0, pb);
    pack_stream(m, b, [&](uint64_t i) { return (uint64_t)(U)((U)x[i] - (U)mn); }, &o.b[off]);
}

// ------------------------------------------------------------------ dictionary + BP
// The sorted distinct values of x[0..m) when there are at most `limit`
// (limit <= 65536), with a rank lookup: an open-addressing hash set of twice
// the limit's size collects them in one pass (no sort of all m rows), then
// only the distinct values are sorted.  Returns false above the limit.
template <class T>
struct DistinctRanks {
    using U = typename std::make_unsigned<T>::type;
    std::vector<T> sorted;           // the distinct values, ascending
    std::vector<T> key;
    std::vector<int32_t> slot;       // -1 = empty, else index into `sorted` (after build)
    uint32_t mask = 0;
    static uint32_t hash(T v) {
        uint64_t z = (uint64_t)(U)v * 0x9E3779B97F4A7C15ull;
        return (uint32_t)(z >> 32);
    }
    bool build(const T* x, uint32_t m, uint32_t limit) {
        uint32_t cap = 16;
        while (cap < 2 * limit) cap <<= 1;
        mask = cap - 1;
        key.assign(cap, T(0));
        slot.assign(cap, -1);
        uint32_t n = 0;
        for (uint32_t i = 0; i < m; i++) {
            const T v = x[i];
            uint32_t h = hash(v) & mask;
            while (slot[h] >= 0 && key[h] != v) h = (h + 1) & mask;
            if (slot[h] < 0) {
                if (n == limit) return false;
                key[h] = v;
                slot[h] = (int32_t)n++;
            }
        }
        sorted.clear();
        for (uint32_t h = 0; h < cap; h++)
            if (slot[h] >= 0) sorted.push_back(key[h]);
        std::sort(sorted.begin(), sorted.end());
        for (uint32_t h = 0; h < cap; h++)
            if (slot[h] >= 0) slot[h] = (int32_t)(std::lower_bound(sorted.begin(), sorted.end(), key[h]) - sorted.begin());
        return true;
    }
    uint32_t rank(T v) const {
        uint32_t h = hash(v) & mask;
        while (key[h] != v || slot[h] < 0) h = (h + 1) & mask;
        return (uint32_t)slot[h];
    }
};

template <class T>
zf_status enc_dict(const T* x, uint32_t m, Out& o) {
    DistinctRanks<T> dr;
    if (!dr.build(x, m, kMaxDict)) return ZF_EINVAL;
    const std::vector<T>& d = dr.sorted;
    uint32_t nd = (uint32_t)d.size();
    uint32_t b = nd ? bits_of(nd - 1) : 0;
    uint64_t pb = packed_bytes(m, b);
    uint64_t dict_bytes = (uint64_t)nd * sizeof(T);
    o.b.assign(align16(align16(kChunkHeader + dict_bytes) + pb), 0);
    ChunkWriter w(o);
    w.header(ZF_DICT_BP, dtype_code<T>(), b, 0, m, nd, 0);
    uint64_t doff = w.section(0, dict_bytes);
    if (nd) memcpy(&o.b[doff], d.data(), dict_bytes);
    uint64_t coff = w.section(1, pb);
    pack_stream(m, b, [&](uint64_t i) { return (uint64_t)dr.rank(x[i]); }, &o.b[coff]);
    return ZF_OK;
}

// ------------------------------------------------------------------ dictionary + ANS
// The chunk's sorted distinct values (at most kAnsMaxSymbols) are symbols,
// coded with range ANS (Duda; byte-wise renormalization, states in
// [kAnsL, 256 kAnsL)): encoding symbol s with frequency f and cumulative
// frequency c out of M = 2^kAnsScale maps x to (x / f) * M + x % f + c after
// emitting low bytes while x >= (kAnsL / M) * 256 * f.  Every kAnsStream rows
// form a stream coded from its last row to its first from x = kAnsL and
// stored as the final state (4 bytes) followed by the emitted bytes, the last
// emitted first.  Frequencies: max(1, count * M / n), a shortfall to the most
// frequent symbol (the first on a tie), an excess taken one at a time from
// the largest frequency above 1 (the first on a tie).  Sections: s0 = values,
// s1 = u16 frequencies (padded to 4 bytes) then u32 stream starts and end,
// s2 = streams.
template <class T>
zf_status enc_ans(const T* x, uint32_t m, uint32_t L, Out& o) {
    DistinctRanks<T> dr;
    if (!dr.build(x, m, kAnsMaxSymbols)) return ZF_EINVAL;
    const std::vector<T>& d = dr.sorted;
    const uint32_t nd = (uint32_t)d.size(), K = (m + L - 1) / L;
    std::vector<uint32_t> sym(m), cnt(nd, 0), f(nd, 0), c(nd, 0);
    for (uint32_t i = 0; i < m; i++) {
        sym[i] = dr.rank(x[i]);
        cnt[sym[i]]++;
    }
    if (nd) {
        uint64_t total = 0;
        for (uint32_t k = 0; k < nd; k++) {
            f[k] = std::max<uint32_t>(1, (uint32_t)((uint64_t)cnt[k] * kAnsM / m));
            total += f[k];
        }
        if (total < kAnsM) {
            const uint32_t top = (uint32_t)(std::max_element(cnt.begin(), cnt.end()) - cnt.begin());  // first maximum
            f[top] += (uint32_t)(kAnsM - total);
        }
        for (; total > kAnsM; total--) {
            uint32_t top = nd;
            for (uint32_t k = 0; k < nd; k++)
                if (f[k] > 1 && (top == nd || f[k] > f[top])) top = k;
            f[top]--;
        }
        for (uint32_t k = 1; k < nd; k++) c[k] = c[k - 1] + f[k - 1];
    }
    // streams, each written back to front into its own buffer
    std::vector<std::vector<uint8_t>> st(K);
    uint64_t sbytes = 0;
    for (uint32_t j = 0; j < K; j++) {
        const uint32_t r0 = j * L, n = std::min(L, m - r0);
        std::vector<uint8_t> rev;
        rev.reserve(2 * n + 8);
        uint32_t s_x = kAnsL;
        for (uint32_t i = n; i-- > 0;) {
            const uint32_t s = sym[r0 + i];
            const uint64_t lim = (uint64_t)(kAnsL >> kAnsScale) * 256u * f[s];
            while (s_x >= lim) {
                rev.push_back((uint8_t)s_x);
                s_x >>= 8;
            }
            s_x = (s_x / f[s]) * kAnsM + s_x % f[s] + c[s];
        }
        auto& out = st[j];
        out.resize(4 + rev.size());
        memcpy(out.data(), &s_x, 4);
        std::copy(rev.rbegin(), rev.rend(), out.begin() + 4);
        sbytes += out.size();
    }
    const uint64_t fbytes = (2ull * nd + 3) / 4 * 4, l0 = (uint64_t)nd * sizeof(T), l1 = fbytes + 4ull * (K + 1);
    o.b.assign(align16(align16(align16(kChunkHeader + l0) + l1) + sbytes), 0);
    ChunkWriter w(o);
    w.header(ZF_ANS, dtype_code<T>(), kAnsScale, 0, m, nd, K);
    o.b[48] = (uint8_t)(31 - __builtin_clz(L));   // log2 of the rows per stream
    const uint64_t s0 = w.section(0, l0), s1 = w.section(1, l1), s2 = w.section(2, sbytes);
    if (nd) memcpy(&o.b[s0], d.data(), l0);
    for (uint32_t k = 0; k < nd; k++) {
        const uint16_t v = (uint16_t)f[k];
        memcpy(&o.b[s1 + 2ull * k], &v, 2);
    }
    uint64_t pos = 0;
    for (uint32_t j = 0; j < K; j++) {
        o.put32(s1 + fbytes + 4ull * j, (uint32_t)pos);
        memcpy(o.b.data() + s2 + pos, st[j].data(), st[j].size());
        pos += st[j].size();
    }
    o.put32(s1 + fbytes + 4ull * K, (uint32_t)pos);
    return ZF_OK;
}

// ------------------------------------------------------------------ delta + BP
template <class T>
void enc_delta(const T* x, uint32_t m, Out& o) {
    using U = typename std::make_unsigned<T>::type;
    uint32_t nb = (m + kDeltaBlock - 1) / kDeltaBlock;
    struct Blk { T base, min_d; uint32_t b; uint64_t poff, len; };
    std::vector<Blk> blk(nb);
    uint64_t payload = 0;
    for (uint32_t k = 0; k < nb; k++) {
        uint32_t r0 = k * kDeltaBlock, mk = std::min(kDeltaBlock, m - r0);
        const T* y = x + r0;
        T min_d = 0;
        for (uint32_t j = 1; j < mk; j++) {
            T d = (T)(U)((U)y[j] - (U)y[j - 1]);
            if (j == 1 || d < min_d) min_d = d;
        }
        U umax = 0;
        for (uint32_t j = 1; j < mk; j++) {
            U u = (U)((U)y[j] - (U)y[j - 1]) - (U)min_d;
            umax = std::max(umax, u);
        }
        uint32_t b = bits_of((uint64_t)umax);
        uint64_t len = align16(packed_bytes(mk, b));
        blk[k] = {y[0], min_d, b, payload, len};
        payload += len;
    }
    uint64_t table = (uint64_t)nb * kDeltaEntry;
    o.b.assign(align16(align16(kChunkHeader + table) + payload), 0);
    ChunkWriter w(o);
    w.header(ZF_DELTA_BP, dtype_code<T>(), 0, 0, m, nb, 0);
    uint64_t toff = w.section(0, table);
    uint64_t poff = w.section(1, payload);
    for (uint32_t k = 0; k < nb; k++) {
        uint8_t* e = &o.b[toff + (uint64_t)k * kDeltaEntry];
        int64_t base = blk[k].base, min_d = blk[k].min_d;
        uint32_t po = (uint32_t)blk[k].poff;
        memcpy(e, &base, 8);
        memcpy(e + 8, &min_d, 8);
        memcpy(e + 16, &po, 4);
        e[20] = (uint8_t)blk[k].b;
        const T* y = x + (uint64_t)k * kDeltaBlock;
        uint32_t mk = std::min(kDeltaBlock, m - k * kDeltaBlock);
        U md = (U)blk[k].min_d;
        pack_stream(mk, blk[k].b, [&](uint64_t j) {
            return j == 0 ? 0ull : (uint64_t)(U)((U)((U)y[j] - (U)y[j - 1]) - md);
        }, &o.b[poff + blk[k].poff]);
    }
}

// ------------------------------------------------------------------ RLE
template <class T>
void enc_rle(const T* x, uint32_t m, Out& o) {
    uint32_t R = 0;
    for (uint32_t i = 0; i < m; i++) R += (i == 0 || x[i] != x[i - 1]);
    uint32_t nt = (m + kRleDirRows - 1) / kRleDirRows;
    uint64_t vb = (uint64_t)R * sizeof(T), lb = 4ull * R, db = 8ull * nt;
    o.b.assign(align16(align16(align16(align16(kChunkHeader) + vb) + lb) + db), 0);
    ChunkWriter w(o);
    w.header(ZF_RLE, dtype_code<T>(), 0, 0, m, R, 0);
    uint64_t voff = w.section(0, vb), loff = w.section(1, lb), doff = w.section(2, db);
    T* vals = reinterpret_cast<T*>(&o.b[voff]);
    uint32_t* lens = reinterpret_cast<uint32_t*>(&o.b[loff]);
    uint32_t* dir = reinterpret_cast<uint32_t*>(&o.b[doff]);
    uint32_t r = 0, start = 0;
    for (uint32_t i = 0; i < m; i++) {
        if (i > 0 && x[i] != x[i - 1]) {
            lens[r++] = i - start;
            start = i;
        }
        if (i == start) vals[r] = x[i];
        if (i % kRleDirRows == 0) {
            dir[2 * (i / kRleDirRows)] = r;
            dir[2 * (i / kRleDirRows) + 1] = i - start;
        }
    }
    if (m) lens[r] = m - start;
}

// ------------------------------------------------------------------ LZ77
uint32_t leb128(uint8_t* p, uint32_t v) {
    uint32_t n = 0;
    do {
        uint8_t c = v & 0x7F;
        v >>= 7;
        p[n++] = c | (v ? 0x80 : 0);
    } while (v);
    return n;
}

// Greedy LZ77 over one block: a hash of 4 bytes indexes the most recent
// position; every position, including those inside a match, is inserted.
// Output streams: lengths (LEB128 literal length of each token, and between
// tokens the match length - 4), u16 offsets, literal bytes.
void enc_lz(const uint8_t* s, uint32_t m, Out& o) {
    constexpr int HB = 15;
    std::vector<int32_t> table(1u << HB, -1);
    std::vector<uint8_t> lens, offs, lit;
    lens.reserve(m / 4 + 16);
    offs.reserve(m / 4 + 16);
    lit.reserve(m + 16);
    auto hash = [&](uint32_t p) {
        uint32_t v;
        memcpy(&v, s + p, 4);
        return (v * 2654435761u) >> (32 - HB);
    };
    uint8_t tmp[16];
    uint32_t ntok = 0, pos = 0, lit_start = 0;
    while (pos + kLzMinMatch <= m) {
        uint32_t h = hash(pos);
        int32_t cand = table[h];
        table[h] = (int32_t)pos;
        uint32_t len = 0;
        if (cand >= 0 && pos - (uint32_t)cand <= kLzMaxOffset && memcmp(s + cand, s + pos, kLzMinMatch) == 0) {
            len = kLzMinMatch;
            while (pos + len < m && s[cand + len] == s[pos + len]) len++;
        }
        if (!len) {
            pos++;
            continue;
        }
        lens.insert(lens.end(), tmp, tmp + leb128(tmp, pos - lit_start));
        lit.insert(lit.end(), s + lit_start, s + pos);
        lens.insert(lens.end(), tmp, tmp + leb128(tmp, len - kLzMinMatch));
        const uint32_t off = pos - (uint32_t)cand;
        offs.push_back((uint8_t)off);
        offs.push_back((uint8_t)(off >> 8));
        ntok++;
        for (uint32_t q = pos + 1; q < pos + len && q + kLzMinMatch <= m; q++) table[hash(q)] = (int32_t)q;
        pos += len;
        lit_start = pos;
    }
    lens.insert(lens.end(), tmp, tmp + leb128(tmp, m - lit_start));
    lit.insert(lit.end(), s + lit_start, s + m);
    ntok++;
    if (lens.size() + offs.size() + lit.size() >= m) {
        o.b.assign(align16(kChunkHeader + m), 0);
        ChunkWriter w(o);
        w.header(ZF_LZ77, ZF_BYTES, 0, 1, m, 0, 0);
        uint64_t off = w.section(0, m);
        if (m) memcpy(&o.b[off], s, m);
        return;
    }
    o.b.assign(align16(align16(align16(kChunkHeader + lens.size()) + offs.size()) + lit.size()), 0);
    ChunkWriter w(o);
    w.header(ZF_LZ77, ZF_BYTES, 0, 0, m, ntok, 0);
    uint64_t a = w.section(0, lens.size());
    memcpy(&o.b[a], lens.data(), lens.size());
    uint64_t b = w.section(1, offs.size());
    if (!offs.empty()) memcpy(&o.b[b], offs.data(), offs.size());
    uint64_t c = w.section(2, lit.size());
    if (!lit.empty()) memcpy(&o.b[c], lit.data(), lit.size());
}

// ------------------------------------------------------------------ column assembly
struct PartSpec {
    int scheme, dtype;
    const uint8_t* data;
    uint64_t n;
    uint32_t chunk_rows;
    const int32_t* offsets = nullptr;   // string dictionary: row starts (nrows + 1 entries)
    uint64_t nrows = 0;
    uint32_t ans_stream = kAnsStream;   // ANS: rows per independent stream
};

void run_parallel(uint32_t n, const std::function<void(uint32_t)>& f) {
    unsigned nt = std::max(1u, std::min(std::thread::hardware_concurrency(), n));
    std::atomic<uint32_t> next{0};
    auto worker = [&] {
        for (uint32_t i; (i = next.fetch_add(1)) < n;) f(i);
    };
    if (nt <= 1) {
        worker();
        return;
    }
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; t++) th.emplace_back(worker);
    for (auto& t : th) t.join();
}

zf_status encode_part(const PartSpec& p, std::vector<Out>& blobs, std::string* why) {
    uint64_t nch = (p.n + p.chunk_rows - 1) / p.chunk_rows;
    blobs.assign(nch, Out{});
    std::atomic<int> err{ZF_OK};
    uint32_t sz = dtype_size(p.dtype);
    run_parallel((uint32_t)nch, [&](uint32_t c) {
        uint64_t r0 = (uint64_t)c * p.chunk_rows;
        uint32_t m = (uint32_t)std::min<uint64_t>(p.chunk_rows, p.n - r0);
        const uint8_t* x = p.data + r0 * sz;
        Out& o = blobs[c];
        zf_status st = ZF_OK;
        if (p.dtype == ZF_BYTES) {
            if (p.scheme == ZF_LZ77) {
                enc_lz(x, m, o);
            } else if (p.scheme == ZF_STRDICT) {
                // rows that start inside the chunk (offsets are nondecreasing)
                std::vector<uint8_t> row_start((size_t)m + 1, 0);
                const int32_t* q = std::lower_bound(p.offsets, p.offsets + p.nrows + 1, (int64_t)r0,
                                                    [](int32_t a, int64_t v) { return (int64_t)a < v; });
                for (; q < p.offsets + p.nrows + 1 && (uint64_t)*q < r0 + m; q++) row_start[*q - r0] = 1;
                enc_strdict(x, m, row_start, o);
            } else {  // RAW bytes
                o.b.assign(align16(kChunkHeader + m), 0);
                ChunkWriter w(o);
                w.header(ZF_RAW, ZF_BYTES, 0, 0, m, 0, 0);
                uint64_t off = w.section(0, m);
                if (m) memcpy(&o.b[off], x, m);
            }
        } else if (p.dtype == ZF_F64) {
            if (p.scheme == ZF_FLOAT2INT) {
                enc_f2i(reinterpret_cast<const double*>(x), m, o);
            } else {  // RAW doubles
                o.b.assign(align16(kChunkHeader + 8ull * m), 0);
                ChunkWriter w(o);
                w.header(ZF_RAW, ZF_F64, 0, 0, m, 0, 0);
                uint64_t off = w.section(0, 8ull * m);
                if (m) memcpy(&o.b[off], x, 8ull * m);
            }
        } else if (p.dtype == ZF_I32) {
            auto* v = reinterpret_cast<const int32_t*>(x);
            switch (p.scheme) {
            case ZF_RAW: enc_raw(v, m, o); break;
            case ZF_FOR_BP: enc_for(v, m, o); break;
            case ZF_DICT_BP: st = enc_dict(v, m, o); break;
            case ZF_DELTA_BP: enc_delta(v, m, o); break;
            case ZF_RLE: enc_rle(v, m, o); break;
            case ZF_ANS: st = enc_ans(v, m, p.ans_stream, o); break;
            }
        } else {
            auto* v = reinterpret_cast<const int64_t*>(x);
            switch (p.scheme) {
            case ZF_RAW: enc_raw(v, m, o); break;
            case ZF_FOR_BP: enc_for(v, m, o); break;
            case ZF_DICT_BP: st = enc_dict(v, m, o); break;
            case ZF_DELTA_BP: enc_delta(v, m, o); break;
            case ZF_RLE: enc_rle(v, m, o); break;
            case ZF_ANS: st = enc_ans(v, m, p.ans_stream, o); break;
            }
        }
        if (st != ZF_OK) err = st;
    });
    if (err != ZF_OK) {
        if (why) *why = "scheme does not fit the column (dictionary above 65,536 entries, or ANS above 256 values)";
        return (zf_status)err.load();
    }
    return ZF_OK;
}

uint64_t part_size(const std::vector<Out>& blobs) {
    uint64_t s = kColHeader + (uint64_t)kDirEntry * blobs.size();
    for (auto& b : blobs) s += b.b.size();
    return s;
}

void write_part(const PartSpec& p, const std::vector<Out>& blobs, uint8_t* dst, uint32_t flags) {
    uint64_t nch = blobs.size();
    uint64_t total = part_size(blobs);
    memset(dst, 0, kColHeader + kDirEntry * nch);
    uint32_t magic = kColMagic;
    uint16_t ver = 1;
    memcpy(dst, &magic, 4);
    memcpy(dst + 4, &ver, 2);
    dst[6] = (uint8_t)p.scheme;
    dst[7] = (uint8_t)p.dtype;
    uint32_t n32 = (uint32_t)nch;
    memcpy(dst + 8, &n32, 4);
    memcpy(dst + 12, &p.chunk_rows, 4);
    memcpy(dst + 16, &p.n, 8);
    uint64_t raw = p.n * dtype_size(p.dtype);
    memcpy(dst + 24, &raw, 8);
    memcpy(dst + 32, &total, 8);
    memcpy(dst + 40, &flags, 4);
    std::vector<uint64_t> offs(nch);
    uint64_t pos = kColHeader + kDirEntry * nch;
    for (uint64_t c = 0; c < nch; c++) {
        offs[c] = pos;
        uint8_t* d = dst + kColHeader + kDirEntry * c;
        uint64_t len = blobs[c].b.size(), r0 = c * p.chunk_rows;
        uint32_t m = (uint32_t)std::min<uint64_t>(p.chunk_rows, p.n - r0);
        memcpy(d, &pos, 8);
        memcpy(d + 8, &len, 8);
        memcpy(d + 16, &r0, 8);
        memcpy(d + 24, &m, 4);
        pos += len;
    }
    run_parallel((uint32_t)nch, [&](uint32_t c) {
        if (!blobs[c].b.empty()) memcpy(dst + offs[c], blobs[c].b.data(), blobs[c].b.size());
    });
}

bool scheme_fits(int scheme, int dtype) {
    if (dtype == ZF_BYTES) return scheme == ZF_RAW || scheme == ZF_LZ77 || scheme == ZF_STRDICT;
    if (dtype == ZF_F64) return scheme == ZF_RAW || scheme == ZF_FLOAT2INT;
    if (dtype != ZF_I32 && dtype != ZF_I64) return false;
    return (scheme >= ZF_RAW && scheme <= ZF_RLE) || scheme == ZF_ANS;
}

}  // namespace

// Allocate host memory for serialized bytes: pinned when a CUDA device is
// present, plain memory when the machine has none (host-only use).
static zf_status alloc_host(zf_compressed* c, uint64_t len) {
    void* p = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
        cudaError_t e = cudaHostAlloc(&p, std::max<uint64_t>(len, 16), cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return ZF_ENOMEM;
        }
        c->pinned = true;
    } else {
        cudaGetLastError();
        p = malloc(std::max<uint64_t>(len, 16));
        if (!p) return ZF_ENOMEM;
        c->pinned = false;
    }
    c->host = (uint8_t*)p;
    c->len = len;
    return ZF_OK;
}

void free_compressed(zf_compressed* c) {
    if (!c) return;
    if (c->host) {
        if (c->pinned) cudaFreeHost(c->host);
        else free(c->host);
    }
    delete c;
}

zf_status encode_column(const zf_plan_t& plan, const zf_column& col, zf_compressed** out, std::string* why) {
    int dt = col.dtype;
    if (dt != ZF_I32 && dt != ZF_I64 && dt != ZF_BYTES && dt != ZF_F64) return ZF_EINVAL;
    if (col.n && !col.data && !(dt == ZF_BYTES && col.offsets)) return ZF_EINVAL;
    std::vector<PartSpec> specs;
    if (dt == ZF_BYTES) {
        if (!col.offsets) return ZF_EINVAL;
        if (col.offsets[0] != 0) return ZF_EINVAL;
        for (uint64_t i = 0; i < col.n; i++)
            if (col.offsets[i + 1] < col.offsets[i]) return ZF_EINVAL;
        int bs = (plan.scheme == ZF_RAW || plan.scheme == ZF_STRDICT) ? plan.scheme : ZF_LZ77;
        int os = plan.offsets_scheme < 0 ? ZF_DELTA_BP : plan.offsets_scheme;
        if (!scheme_fits(os, ZF_I32)) return ZF_EINVAL;
        uint32_t cb = kLzBlock;
        if (bs == ZF_STRDICT) {
            cb = plan.chunk_rows;
            if (cb == 0 || cb % kLzBlock || cb > kStrChunkMax) {
                if (why) *why = "string-dictionary chunks are a multiple of 65536 bytes, at most 2^26";
                return ZF_EINVAL;
            }
        }
        uint64_t nbytes = (uint64_t)(uint32_t)col.offsets[col.n];
        PartSpec bytes{bs, ZF_BYTES, (const uint8_t*)col.data, nbytes, cb};
        bytes.offsets = col.offsets;
        bytes.nrows = col.n;
        specs.push_back(bytes);
        specs.push_back({os, ZF_I32, (const uint8_t*)col.offsets, col.n + 1, 65536});
    } else {
        if (!scheme_fits(plan.scheme, dt) || plan.scheme == ZF_LZ77) return ZF_EINVAL;
        uint32_t cr = plan.chunk_rows ? plan.chunk_rows : (1u << 20);
        if (cr % 1024 != 0) {
            if (why) *why = "chunk_rows must be a multiple of 1024";
            return ZF_EINVAL;
        }
        specs.push_back({plan.scheme, dt, (const uint8_t*)col.data, col.n, cr});
        if (plan.scheme == ZF_ANS) {
            const uint32_t L = plan.ans_stream_rows ? plan.ans_stream_rows : kAnsStream;
            if ((L & (L - 1)) || L < (1u << kAnsLogMin) || L > (1u << kAnsLogMax)) {
                if (why) *why = "ANS streams are a power of two of 32..4096 rows";
                return ZF_EINVAL;
            }
            specs.back().ans_stream = L;
        }
    }
    std::vector<std::vector<Out>> blobs(specs.size());
    uint64_t total = 0;
    for (size_t p = 0; p < specs.size(); p++) {
        zf_status st = encode_part(specs[p], blobs[p], why);
        if (st) return st;
        total += part_size(blobs[p]);
    }
    auto* c = new zf_compressed();
    zf_status st = alloc_host(c, total);
    if (st) {
        delete c;
        return st;
    }
    uint64_t pos = 0;
    for (size_t p = 0; p < specs.size(); p++) {
        write_part(specs[p], blobs[p], c->host + pos, (specs.size() == 2 && p == 0) ? 1u : 0u);
        pos += part_size(blobs[p]);
        std::vector<Out>().swap(blobs[p]);
    }
    st = parse_serialized(c, why);
    if (st) {
        free_compressed(c);
        return st;
    }
    *out = c;
    return ZF_OK;
}

// Warp jobs of a chunk: one per LZ77 block (its own kernel), else one per
// tile_rows rows (bytes for a raw byte chunk).
uint32_t tiles_of(const ChunkInfo& ch, uint32_t tile_rows) {
    if (ch.scheme == ZF_LZ77) return 1;
    if (ch.scheme == ZF_STRDICT) return (ch.units + tile_rows - 1) / tile_rows;   // jobs of tile_rows tokens
    if (ch.scheme == ZF_ANS) {   // 32 streams a job, a chunk's jobs padded to whole CTAs
        const uint32_t jobs = (ch.units + kAnsStreamsPerJob - 1) / kAnsStreamsPerJob;
        return (jobs + kAnsJobsPerCta - 1) / kAnsJobsPerCta * kAnsJobsPerCta;
    }
    return (ch.rows + tile_rows - 1) / tile_rows;
}

// ------------------------------------------------------------------ validation
namespace {
template <class T> T rd(const uint8_t* p) { T v; memcpy(&v, p, sizeof(T)); return v; }

bool fail(std::string* why, const std::string& m) {
    if (why) *why = m;
    return false;
}

bool check_chunk(const uint8_t* c, uint64_t len, int scheme, int dtype, uint32_t rows, uint8_t* bmax,
                 std::string* why) {
    *bmax = 0;
    if (len < kChunkHeader || len % 16) return fail(why, "chunk blob too short or not a multiple of 16");
    if (rd<uint32_t>(c) != kChunkMagic) return fail(why, "bad chunk magic");
    if (c[4] != scheme || c[5] != dtype) return fail(why, "chunk scheme/dtype differ from the column");
    if (rd<uint32_t>(c + 8) != rows) return fail(why, "chunk rows differ from the directory");
    uint32_t b = c[6], n_aux = rd<uint32_t>(c + 12);
    uint32_t off[3], ln[3];
    for (int s = 0; s < 3; s++) {
        off[s] = rd<uint32_t>(c + 24 + 4 * s);
        ln[s] = rd<uint32_t>(c + 36 + 4 * s);
    }
    int nsec = 0;
    switch (scheme) {
    case ZF_RAW: case ZF_FOR_BP: nsec = 1; break;
    case ZF_DICT_BP: nsec = 2; break;
    case ZF_DELTA_BP: nsec = 2; break;
    case ZF_RLE: nsec = 3; break;
    case ZF_LZ77: nsec = (c[7] & 1) ? 1 : 3; break;
    case ZF_FLOAT2INT: nsec = 3; break;
    case ZF_STRDICT: nsec = 3; break;
    case ZF_ANS: nsec = 3; break;
    default: return fail(why, "unknown scheme");
    }
    for (int s = 0; s < nsec; s++)
        if (off[s] < kChunkHeader || off[s] % 16 || (uint64_t)off[s] + ln[s] > len)
            return fail(why, "section outside the blob or misaligned");
    uint32_t sz = dtype_size(dtype), wd = 8 * sz;
    switch (scheme) {
    case ZF_RAW:
        if (ln[0] != (uint64_t)rows * sz) return fail(why, "raw section length");
        break;
    case ZF_FOR_BP:
        if (b > wd || ln[0] != packed_bytes(rows, b)) return fail(why, "FOR width or payload length");
        *bmax = (uint8_t)b;
        break;
    case ZF_DICT_BP:
        if (n_aux > kMaxDict || (rows && n_aux == 0) || ln[0] != (uint64_t)n_aux * sz ||
            b != (n_aux ? bits_of(n_aux - 1) : 0) || ln[1] != packed_bytes(rows, b))
            return fail(why, "dictionary header");
        *bmax = (uint8_t)b;
        break;
    case ZF_DELTA_BP: {
        uint32_t nb = (rows + kDeltaBlock - 1) / kDeltaBlock;
        if (n_aux != nb || ln[0] != (uint64_t)nb * kDeltaEntry) return fail(why, "delta block table");
        for (uint32_t k = 0; k < nb; k++) {
            const uint8_t* e = c + off[0] + (uint64_t)k * kDeltaEntry;
            uint32_t po = rd<uint32_t>(e + 16), bk = e[20];
            uint32_t mk = std::min(kDeltaBlock, rows - k * kDeltaBlock);
            if (bk > wd || po % 16 || (uint64_t)po + align16(packed_bytes(mk, bk)) > ln[1])
                return fail(why, "delta block entry");
            *bmax = (uint8_t)std::max<uint32_t>(*bmax, bk);
        }
        break;
    }
    case ZF_RLE:
        if (n_aux > rows || (rows && !n_aux) || ln[0] != (uint64_t)n_aux * sz || ln[1] != 4ull * n_aux ||
            ln[2] != 8ull * ((rows + kRleDirRows - 1) / kRleDirRows))
            return fail(why, "RLE sections");
        break;
    case ZF_FLOAT2INT: {
        if (b > 64 || c[48] > kF2IMaxExp || n_aux > rows || ln[0] != packed_bytes(rows, b) ||
            ln[1] != 4ull * n_aux || ln[2] != 8ull * n_aux)
            return fail(why, "Float2Int sections");
        // exception rows strictly increasing and inside the chunk
        for (uint32_t k = 0; k < n_aux; k++) {
            const uint32_t r = rd<uint32_t>(c + off[1] + 4ull * k);
            if (r >= rows || (k && r <= rd<uint32_t>(c + off[1] + 4ull * (k - 1))))
                return fail(why, "Float2Int exception rows");
        }
        *bmax = (uint8_t)b;
        break;
    }
    case ZF_ANS: {
        const uint64_t K = rd<uint64_t>(c + 16), fb = (2ull * n_aux + 3) / 4 * 4;
        const uint32_t lg = c[48];
        if (lg < kAnsLogMin || lg > kAnsLogMax) return fail(why, "ANS stream length");
        const uint32_t L = 1u << lg;
        if (b != kAnsScale || n_aux == 0 || n_aux > kAnsMaxSymbols || ln[0] != (uint64_t)n_aux * sz ||
            K != (rows + L - 1) / L || ln[1] != fb + 4 * (K + 1))
            return fail(why, "ANS sections");
        // frequencies of at least 1 that fill M; streams of at least the 4 state bytes that fill s2
        uint32_t total = 0;
        for (uint32_t k = 0; k < n_aux; k++) {
            const uint32_t fk = rd<uint16_t>(c + off[1] + 2ull * k);
            if (fk == 0) return fail(why, "ANS frequency");
            total += fk;
        }
        if (total != kAnsM) return fail(why, "ANS frequencies do not fill M");
        const uint8_t* st = c + off[1] + fb;
        if (rd<uint32_t>(st) != 0 || rd<uint32_t>(st + 4 * K) != ln[2]) return fail(why, "ANS stream table");
        for (uint64_t j = 0; j < K; j++)
            if (rd<uint32_t>(st + 4 * (j + 1)) < rd<uint32_t>(st + 4 * j) + 4ull) return fail(why, "ANS stream");
        break;
    }
    case ZF_STRDICT: {
        const uint64_t T = rd<uint64_t>(c + 16), ntiles = (T + kStrTile - 1) / kStrTile;
        if (n_aux == 0 || n_aux > kStrDictMax || b != bits_of(n_aux - 1) || T > rows || (rows && T == 0) ||
            ln[0] != 4ull * (n_aux + 1 + ntiles) || ln[2] != packed_bytes(T, b))
            return fail(why, "string-dictionary sections");
        // dictionary entries of 1..kStrTokenMax bytes, in order, filling s1
        const uint8_t* d = c + off[0];
        if (rd<uint32_t>(d) != 0 || rd<uint32_t>(d + 4ull * n_aux) != ln[1])
            return fail(why, "string-dictionary offsets");
        for (uint32_t k = 0; k < n_aux; k++) {
            const uint32_t a0 = rd<uint32_t>(d + 4ull * k), a1 = rd<uint32_t>(d + 4ull * (k + 1));
            if (a1 <= a0 || a1 - a0 > kStrTokenMax) return fail(why, "string-dictionary entry");
        }
        // tile starts: the first is 0, then nondecreasing and inside the chunk
        for (uint64_t j = 0; j < ntiles; j++) {
            const uint32_t t0 = rd<uint32_t>(d + 4ull * (n_aux + 1 + j));
            if ((j == 0 && t0 != 0) || t0 > rows || (j && t0 < rd<uint32_t>(d + 4ull * (n_aux + j))))
                return fail(why, "string-dictionary tile starts");
        }
        *bmax = (uint8_t)b;
        break;
    }
    case ZF_LZ77:
        if (rows > kLzBlock) return fail(why, "LZ77 block above 64 KiB");
        if ((c[7] & 1) && ln[0] != rows) return fail(why, "raw LZ77 block length");
        if (!(c[7] & 1) && (n_aux == 0 || ln[1] != 2ull * (n_aux - 1) || ln[0] < 2ull * n_aux - 1))
            return fail(why, "LZ77 token streams");
        break;
    }
    return true;
}
}  // namespace

zf_status parse_serialized(zf_compressed* c, std::string* why) {
    c->chunks.clear();
    c->nparts = 0;
    c->raw_bytes = 0;
    uint64_t pos = 0;
    for (int p = 0; p < 2; p++) {
        const uint8_t* h = c->host + pos;
        if (pos + kColHeader > c->len || rd<uint32_t>(h) != kColMagic || rd<uint16_t>(h + 4) != 1) {
            fail(why, "bad column header");
            return ZF_ECORRUPT;
        }
        PartInfo& pi = c->parts[p];
        pi.off = pos;
        pi.scheme = h[6];
        pi.dtype = h[7];
        uint32_t nch = rd<uint32_t>(h + 8);
        pi.chunk_rows = rd<uint32_t>(h + 12);
        pi.n_rows = rd<uint64_t>(h + 16);
        pi.len = rd<uint64_t>(h + 32);
        uint32_t flags = rd<uint32_t>(h + 40);
        if (!scheme_fits(pi.scheme, pi.dtype) || pi.len > c->len - pos ||
            kColHeader + (uint64_t)kDirEntry * nch > pi.len || pi.chunk_rows == 0 ||
            (uint64_t)nch != (pi.n_rows + pi.chunk_rows - 1) / pi.chunk_rows ||
            rd<uint64_t>(h + 24) != pi.n_rows * dtype_size(pi.dtype)) {
            fail(why, "inconsistent column header");
            return ZF_ECORRUPT;
        }
        if (pi.dtype != ZF_BYTES && (pi.chunk_rows % 1024 || pi.chunk_rows > (1u << 30))) {
            fail(why, "chunk_rows must be a multiple of 1024 and at most 2^30");
            return ZF_ECORRUPT;
        }
        if (pi.n_rows > (1ull << 48)) {
            fail(why, "column above 2^48 rows");
            return ZF_ECORRUPT;
        }
        if (pi.dtype == ZF_BYTES && (pi.scheme == ZF_STRDICT
                                         ? (pi.chunk_rows % kLzBlock || pi.chunk_rows > kStrChunkMax)
                                         : pi.chunk_rows != kLzBlock)) {
            fail(why, "byte chunks must be 65536 bytes (string dictionary: a multiple, at most 2^26)");
            return ZF_ECORRUPT;
        }
        pi.first_chunk = (uint32_t)c->chunks.size();
        pi.n_chunks = nch;
        uint64_t expect = kColHeader + (uint64_t)kDirEntry * nch;
        for (uint32_t k = 0; k < nch; k++) {
            const uint8_t* d = h + kColHeader + (uint64_t)kDirEntry * k;
            ChunkInfo ch{};
            ch.off = rd<uint64_t>(d);
            ch.bytes = rd<uint64_t>(d + 8);
            ch.row0 = rd<uint64_t>(d + 16);
            ch.rows = rd<uint32_t>(d + 24);
            if (ch.off != expect || ch.bytes > pi.len - ch.off || ch.row0 != (uint64_t)k * pi.chunk_rows ||
                ch.rows != std::min<uint64_t>(pi.chunk_rows, pi.n_rows - ch.row0)) {
                fail(why, "bad chunk directory entry");
                return ZF_ECORRUPT;
            }
            expect += ch.bytes;
            if (!check_chunk(h + ch.off, ch.bytes, pi.scheme, pi.dtype, ch.rows, &ch.bmax, why)) return ZF_ECORRUPT;
            if (pi.scheme == ZF_STRDICT || pi.scheme == ZF_ANS) ch.units = (uint32_t)rd<uint64_t>(h + ch.off + 16);
            ch.off += pos;
            ch.scheme = (uint8_t)pi.scheme;
            ch.dtype = (uint8_t)pi.dtype;
            ch.part = (uint8_t)p;
            c->chunks.push_back(ch);
        }
        if (expect != pi.len) {
            fail(why, "column length differs from its chunks");
            return ZF_ECORRUPT;
        }
        c->raw_bytes += pi.n_rows * dtype_size(pi.dtype);
        c->nparts = p + 1;
        pos += pi.len;
        if (!(pi.dtype == ZF_BYTES && (flags & 1))) break;
        if (p == 1) break;
    }
    if (c->nparts == 2 && (c->parts[1].dtype != ZF_I32 || c->parts[1].n_rows == 0)) {
        fail(why, "offsets part must be int32");
        return ZF_ECORRUPT;
    }
    if (pos != c->len) {
        fail(why, "trailing bytes after the column");
        return ZF_ECORRUPT;
    }
    return ZF_OK;
}

}  // namespace zf
