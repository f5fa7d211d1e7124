"""Plant one plausible mistake at a time in a copy of the oracle and check
that the pins catch every one (a dropped term, a wrong sign or index, a
transposed operand, a wrong bit order ...).  Each broken copy runs in its own
process so that a crash cannot take the test run down."""
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    "pack_msb_first": ("out[bit / 8] |= (uint8_t)(1u << (bit % 8));", "out[bit / 8] |= (uint8_t)(1u << (7 - bit % 8));"),
    "pack_and_unpack_msb_first": [
        ("out[bit / 8] |= (uint8_t)(1u << (bit % 8));", "out[bit / 8] |= (uint8_t)(1u << (7 - bit % 8));"),
        ("if ((in[bit / 8] >> (bit % 8)) & 1u)", "if ((in[bit / 8] >> (7 - bit % 8)) & 1u)")],
    "for_width_from_max": ("uint32_t b = orc_bits(((uint64_t)mx - (uint64_t)mn) & mask_of(w_));",
                           "uint32_t b = orc_bits((uint64_t)mx & mask_of(w_));"),
    "for_reference_is_max": ("if (i == 0 || v < mn) mn = v;", "if (i == 0 || v > mn) mn = v;"),
    "for_decode_subtracts": ("store_val(out, dtype, i, (ref + orc_unpack_one(s0, i, b)) & msk);",
                             "store_val(out, dtype, i, (ref - orc_unpack_one(s0, i, b)) & msk);"),
    "dict_unsorted": ("qsort(s, m, sizeof(int64_t), cmp_i64);", ""),
    "dict_width_ndict": ("uint32_t b = nd > 0 ? orc_bits(nd - 1) : 0;", "uint32_t b = nd > 0 ? orc_bits(nd) : 0;"),
    "delta_drops_min_d": ("prev = (prev + min_d + orc_unpack_one(s1 + poff, j, bk)) & msk;",
                          "prev = (prev + orc_unpack_one(s1 + poff, j, bk)) & msk;"),
    "delta_transposed_difference": (
        "int64_t d = sext((uint64_t)load_val(x, dtype, r0 + j) - (uint64_t)load_val(x, dtype, r0 + j - 1), wd);\n"
        "                if (j == 1",
        "int64_t d = sext((uint64_t)load_val(x, dtype, r0 + j - 1) - (uint64_t)load_val(x, dtype, r0 + j), wd);\n"
        "                if (j == 1"),
    "delta_base_is_last": ("int64_t base = load_val(x, dtype, r0);", "int64_t base = load_val(x, dtype, r0 + mk - 1);"),
    "rle_count_off_by_one": ("put_u32(p + loff + 4ull * r, i - run_start);", "put_u32(p + loff + 4ull * r, i - run_start + 1);"),
    "rle_directory_skip": ("put_u32(p + doff + 8ull * (i / RLE_DIR_ROWS) + 4, i - run_start);",
                           "put_u32(p + doff + 8ull * (i / RLE_DIR_ROWS) + 4, run_start);"),
    "rle_decode_next_value": ("uint64_t v = (uint64_t)load_val(s0, dtype, r);",
                              "uint64_t v = (uint64_t)load_val(s0, dtype, r + 1 < R ? r + 1 : r);"),
    "lz_offset_off_by_one": ("for (uint32_t k = 0; k < ml; k++) { o[op] = o[op - off]; op++; }",
                             "for (uint32_t k = 0; k < ml; k++) { o[op] = o[op - off + (off > 1)]; op++; }"),
    "lz_min_match_3": ("ml += LZ_MIN_MATCH;", "ml += 3;"),
    "lz_varint_8bit_shift": ("ll |= (uint32_t)(byte & 0x7F) << sh;\n                sh += 7;",
                             "ll |= (uint32_t)(byte & 0x7F) << sh;\n                sh += 8;"),
    "lz_varint_five_bytes": ("if (vp >= l0 || sh > 14) return ORC_ECORRUPT; /* at most 3 bytes */",
                             "if (vp >= l0 || sh > 28) return ORC_ECORRUPT;"),
    "f2i_multiply_by_reciprocal": ("return (double)d / f2i_pow10(e);", "return (double)d * (1.0 / f2i_pow10(e));"),
    "f2i_no_integer_range_check": ("if (d > F2I_DMAX || d < -F2I_DMAX) return ORC_ECORRUPT;", ""),
    "f2i_no_exception_patch": ("            memcpy(&o[pos], &bits, 8);", "            (void)bits;"),
    "f2i_truncates": ("int64_t k = (int64_t)nearbyint(t);", "int64_t k = (int64_t)t;"),
    "f2i_largest_exponent_on_tie": ("if (ex < best_ex) { best_ex = ex; best_e = e; }",
                                    "if (ex <= best_ex) { best_ex = ex; best_e = e; }"),
    "f2i_reference_is_max": ("if (ok[i] && (!have || d[i] < mn)) { mn = d[i]; have = 1; }",
                             "if (ok[i] && (!have || d[i] > mn)) { mn = d[i]; have = 1; }"),
    "lz_no_raw_fallback": ("if ((uint64_t)nl + no + nlit >= m) {", "if (0) {"),
    "ans_renorm_threshold_halved": ("uint64_t xmax = ((uint64_t)(ANS_L >> ANS_SCALE) << 8) * f[s];",
                                    "uint64_t xmax = ((uint64_t)(ANS_L >> ANS_SCALE) << 7) * f[s];"),
    "ans_shortfall_to_last_on_tie": ("            if (cnt[k] > cnt[best]) best = k;",
                                     "            if (cnt[k] >= cnt[best]) best = k;"),
    "ans_decode_cum_off_by_one": ("x = f[sym] * (x >> ANS_SCALE) + slot - cum[sym];",
                                  "x = f[sym] * (x >> ANS_SCALE) + slot - cum[sym] + (sym > 0);"),
    "ans_stream_length_ignored": ("uint32_t L = 1u << lg;", "uint32_t L = 512u;"),
    "ans_encode_drops_remainder": ("x = (x / f[s]) * ANS_M + (x % f[s]) + c[s];", "x = (x / f[s]) * ANS_M + c[s];"),
    "strdict_tokens_cross_rows": ("while (j < m && x[j - 1] != ' ' && !row_start[j] && j - i < STR_TOKEN_MAX) j++;",
                                  "while (j < m && x[j - 1] != ' ' && j - i < STR_TOKEN_MAX) j++;"),
    "strdict_token_cap_65": ("while (j < m && x[j - 1] != ' ' && !row_start[j] && j - i < STR_TOKEN_MAX) j++;",
                             "while (j < m && x[j - 1] != ' ' && !row_start[j] && j - i <= STR_TOKEN_MAX) j++;"),
    "strdict_first_seen_order": ("    qsort(d, n, sizeof(str_tok), cmp_tok);\n", ""),
    "strdict_no_tile_check": (
        "if (t % STR_TILE == 0 && get_u32(s0 + 4ull * (nd + 1 + t / STR_TILE)) != op) return ORC_ECORRUPT;", ""),
    "lz_offset_of_next_token": ("uint32_t off = get_u16(s1 + 2ull * t);", "uint32_t off = get_u16(s1 + 2ull * (t + 1 < n_aux - 1 ? t + 1 : t));"),
}

RUNNER = r"""
import sys
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import oracle
from oracle_pins import PINS
orc = oracle.Oracle({so!r})
failed = []
for p in PINS:
    try:
        p(orc)
    except Exception as e:
        failed.append(p.__name__)
print("CAUGHT_BY", ",".join(failed))
"""


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    src = open(os.path.join(ROOT, "oracle", "zf_oracle.c")).read()
    subs = MUTANTS[name]
    if isinstance(subs, tuple):
        subs = [subs]
    for old, new in subs:
        assert src.count(old) >= 1, f"mutation site not found: {old[:60]}"
        src = src.replace(old, new, 1)
    c = tmp_path / "mut.c"
    c.write_text(src)
    so = oracle.build(force=True, src=str(c), out=str(tmp_path / "libmut.so"))
    code = RUNNER.format(root=ROOT, tests=os.path.join(ROOT, "tests"), so=so)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    caught = [l for l in r.stdout.splitlines() if l.startswith("CAUGHT_BY")]
    # a crash of the broken copy also counts as caught
    assert r.returncode != 0 or (caught and caught[0] != "CAUGHT_BY "), (name, r.stdout[-500:], r.stderr[-500:])
