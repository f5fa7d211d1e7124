// zf_features.cpp -- the 32 column statistics the learned selector reads.
//
// The statistics describe what each scheme of Section 2.1 exploits: value
// range (bit-packing / FOR), distinct values (dictionary), runs (RLE),
// differences (delta), byte repetition (LZ77).  They are computed on a
// sample: the whole column up to 262,144 rows (bytes for string columns),
// else 64 windows of 4,096 consecutive rows starting at
// floor(i * (n - 4096) / 63), i = 0..63.  Pairs, runs and blocks never
// cross a window.
//
// Integer columns (S sampled values v, W windows, P = S - W pairs, size =
// value bytes; bits(x) = bit length; d = v[i] - v[i-1] wrapping):
//   f0..f2  one-hot dtype (int32, int64, bytes)
//   f3  log2(n + 1) / 32            f4  log2(raw bytes + 1) / 40
//   f5  bits(max - min) / 64        f6  log2(D + 1) / 20, D distinct values
//   f7  D / S                       f8  log2(S / R) / 16, R runs
//   f9  runs of length 1 / R        f10 #(v[i] >= v[i-1]) / P
//   f11 #(v[i] > v[i-1]) / P        f12 bits(max d - min d) / 64
//   f13 mean over 1024-row blocks of bits(max d - min d) / 64
//   f14 mean over windows of bits(max - min) / 64
//   f15 entropy of values (bits) / 20     f16 entropy of d / 20
//   f17 top-1 value share           f18 top-8 value share
//   f19 share of zeros              f20 share of negatives
//   f21, f22 mean and population std of log2(|v| + 1), / 64
//   f23 min(1, R (size + 4) / (S size))   f24 f14 * 64 / (8 size)
//   f25 min(1, (D size + S bits(D - 1) / 8) / (S size))   f26 f13 * 64 / (8 size)
//   f27..f30 0
// String columns (n rows, B bytes; sampled bytes as above):
//   f0..f4 as above (rows, bytes), f5..f26 0,
//   f27 log2(B / max(n, 1) + 1) / 16    f28 byte entropy / 8
//   f29 share of 4-byte windows already seen earlier in their window
//   f30 distinct bytes / 256
// f31 = 1.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "zf_internal.h"

namespace {

constexpr uint64_t kSampleWhole = 262144;
constexpr uint64_t kWindow = 4096;
constexpr uint64_t kWindows = 64;

struct Window {
    uint64_t start, len;
};

std::vector<Window> windows_of(uint64_t n) {
    std::vector<Window> w;
    if (n <= kSampleWhole) {
        if (n) w.push_back({0, n});
        return w;
    }
    for (uint64_t i = 0; i < kWindows; i++) w.push_back({i * (n - kWindow) / (kWindows - 1), kWindow});
    return w;
}

uint32_t bits64(uint64_t x) { return zf::bits_of(x); }

template <class K>
double entropy_of(const std::unordered_map<K, uint64_t>& cnt, uint64_t total) {
    double h = 0;
    for (auto& kv : cnt) {
        const double p = (double)kv.second / (double)total;
        h -= p * std::log2(p);
    }
    return h;
}

template <class T>
void int_features(const T* x, uint64_t n, double* f) {
    const double size = sizeof(T);
    const std::vector<Window> ws = windows_of(n);
    uint64_t S = 0, P = 0, R = 0, runs1 = 0, ge = 0, gt = 0, zeros = 0, neg = 0;
    int64_t mn = 0, mx = 0, dmin = 0, dmax = 0;
    bool have = false, have_d = false;
    double wsum = 0, bsum = 0;
    uint64_t nblocks = 0;
    double lsum = 0, lsq = 0;
    std::unordered_map<int64_t, uint64_t> vc, dc;
    for (const Window& w : ws) {
        int64_t wmn = 0, wmx = 0;
        uint64_t run_len = 0;
        int64_t bdmin = 0, bdmax = 0;
        bool bhave = false;
        for (uint64_t k = 0; k < w.len; k++) {
            const int64_t v = (int64_t)x[w.start + k];
            S++;
            if (!have || v < mn) mn = v;
            if (!have || v > mx) mx = v;
            have = true;
            if (k == 0 || v < wmn) wmn = v;
            if (k == 0 || v > wmx) wmx = v;
            vc[v]++;
            zeros += v == 0;
            neg += v < 0;
            const uint64_t mag = v < 0 ? (uint64_t)0 - (uint64_t)v : (uint64_t)v;
            const double l = std::log2((double)mag + 1.0);
            lsum += l;
            lsq += l * l;
            if (k % 1024 == 0) {
                if (k) {
                    bsum += bhave ? bits64((uint64_t)bdmax - (uint64_t)bdmin) : 0;
                    nblocks++;
                }
                bhave = false;
            }
            if (k == 0) {
                run_len = 1;
                continue;
            }
            const int64_t prev = (int64_t)x[w.start + k - 1];
            const int64_t d = (int64_t)((uint64_t)v - (uint64_t)prev);
            P++;
            ge += v >= prev;
            gt += v > prev;
            if (!have_d || d < dmin) dmin = d;
            if (!have_d || d > dmax) dmax = d;
            have_d = true;
            dc[d]++;
            if (k % 1024 != 0) {
                if (!bhave || d < bdmin) bdmin = d;
                if (!bhave || d > bdmax) bdmax = d;
                bhave = true;
            }
            if (v != prev) {
                R++;
                runs1 += run_len == 1;
                run_len = 1;
            } else {
                run_len++;
            }
        }
        if (w.len) {
            R++;
            runs1 += run_len == 1;
            bsum += bhave ? bits64((uint64_t)bdmax - (uint64_t)bdmin) : 0;
            nblocks++;
            wsum += bits64((uint64_t)wmx - (uint64_t)wmn);
        }
    }
    if (!S) return;
    const uint64_t D = vc.size();
    std::vector<uint64_t> counts;
    counts.reserve(D);
    for (auto& kv : vc) counts.push_back(kv.second);
    std::sort(counts.begin(), counts.end(), std::greater<uint64_t>());
    uint64_t top8 = 0;
    for (size_t i = 0; i < counts.size() && i < 8; i++) top8 += counts[i];
    const double Sd = (double)S;
    f[5] = bits64((uint64_t)mx - (uint64_t)mn) / 64.0;
    f[6] = std::log2((double)D + 1.0) / 20.0;
    f[7] = (double)D / Sd;
    f[8] = std::log2(Sd / (double)R) / 16.0;
    f[9] = (double)runs1 / (double)R;
    f[10] = P ? (double)ge / (double)P : 0.0;
    f[11] = P ? (double)gt / (double)P : 0.0;
    f[12] = have_d ? bits64((uint64_t)dmax - (uint64_t)dmin) / 64.0 : 0.0;
    f[13] = nblocks ? bsum / (double)nblocks / 64.0 : 0.0;
    f[14] = wsum / (double)ws.size() / 64.0;
    f[15] = entropy_of(vc, S) / 20.0;
    f[16] = P ? entropy_of(dc, P) / 20.0 : 0.0;
    f[17] = (double)counts[0] / Sd;
    f[18] = (double)top8 / Sd;
    f[19] = (double)zeros / Sd;
    f[20] = (double)neg / Sd;
    const double mean = lsum / Sd;
    f[21] = mean / 64.0;
    f[22] = std::sqrt(std::max(0.0, lsq / Sd - mean * mean)) / 64.0;
    f[23] = std::min(1.0, (double)R * (size + 4.0) / (Sd * size));
    f[24] = f[14] * 64.0 / (8.0 * size);
    f[25] = std::min(1.0, ((double)D * size + Sd * (double)bits64(D - 1) / 8.0) / (Sd * size));
    f[26] = f[13] * 64.0 / (8.0 * size);
}

void byte_features(const uint8_t* s, uint64_t nbytes, uint64_t rows, double* f) {
    const std::vector<Window> ws = windows_of(nbytes);
    uint64_t cnt[256] = {0};
    uint64_t S = 0, rep = 0, grams = 0;
    for (const Window& w : ws) {
        std::unordered_set<uint32_t> seen;
        for (uint64_t k = 0; k < w.len; k++) {
            cnt[s[w.start + k]]++;
            S++;
            if (k + 4 <= w.len) {
                uint32_t g;
                memcpy(&g, s + w.start + k, 4);
                grams++;
                rep += !seen.insert(g).second;
            }
        }
    }
    f[27] = std::log2((double)nbytes / (double)std::max<uint64_t>(rows, 1) + 1.0) / 16.0;
    double h = 0;
    uint32_t distinct = 0;
    for (int b = 0; b < 256; b++)
        if (cnt[b]) {
            const double p = (double)cnt[b] / (double)S;
            h -= p * std::log2(p);
            distinct++;
        }
    f[28] = S ? h / 8.0 : 0.0;
    f[29] = grams ? (double)rep / (double)grams : 0.0;
    f[30] = distinct / 256.0;
}

}  // namespace

extern "C" zf_status zf_column_features(const zf_column* col, float* out) {
    if (!col || !out) return ZF_EINVAL;
    double f[32] = {0};
    const uint64_t n = col->n;
    if (col->dtype == ZF_I32 || col->dtype == ZF_I64) {
        if (n && !col->data) return ZF_EINVAL;
        const double size = col->dtype == ZF_I64 ? 8.0 : 4.0;
        f[col->dtype == ZF_I32 ? 0 : 1] = 1.0;
        f[3] = std::log2((double)n + 1.0) / 32.0;
        f[4] = std::log2((double)n * size + 1.0) / 40.0;
        if (col->dtype == ZF_I32) int_features((const int32_t*)col->data, n, f);
        else int_features((const int64_t*)col->data, n, f);
    } else if (col->dtype == ZF_BYTES) {
        if (!col->offsets) return ZF_EINVAL;
        const uint64_t nbytes = (uint64_t)(uint32_t)col->offsets[n];
        if (nbytes && !col->data) return ZF_EINVAL;
        f[2] = 1.0;
        f[3] = std::log2((double)n + 1.0) / 32.0;
        f[4] = std::log2((double)nbytes + 1.0) / 40.0;
        byte_features((const uint8_t*)col->data, nbytes, n, f);
    } else {
        return ZF_EINVAL;
    }
    f[31] = 1.0;
    for (int i = 0; i < 32; i++) out[i] = (float)f[i];
    return ZF_OK;
}
