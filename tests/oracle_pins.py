"""Pins of the CPU oracle: facts fixed by the paper's definitions and by
mathematics, not by the oracle itself.

Each ``pin_*`` function takes a loaded oracle and raises AssertionError when
the oracle breaks the fact.  ``test_oracle_pins.py`` runs them on the oracle;
``test_oracle_mutants.py`` runs them on copies of the oracle with a planted
mistake and checks that every mistake is caught.
"""
from __future__ import annotations

import os
import struct

import numpy as np

import oracle as O
import zf_workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
I32_MIN, I32_MAX = -(1 << 31), (1 << 31) - 1
I64_MIN, I64_MAX = -(1 << 63), (1 << 63) - 1


# ---------------------------------------------------------------------------
# a reader of the chunk layout, typed in from the format description
# ---------------------------------------------------------------------------
def parse_chunk(blob: bytes) -> dict:
    magic, scheme, dtype, bw, flags, rows, n_aux, ref = struct.unpack_from("<IBBBBIIq", blob, 0)
    offs = struct.unpack_from("<3I", blob, 24)
    lens = struct.unpack_from("<3I", blob, 36)
    assert magic == 0x4B48435A
    secs = [bytes(blob[o:o + l]) if (o or l) else b"" for o, l in zip(offs, lens)]
    return dict(scheme=scheme, dtype=dtype, bw=bw, flags=flags, rows=rows, n_aux=n_aux, ref=ref,
                offs=offs, lens=lens, secs=secs, b48=blob[48])


def chunks_of(orc, buf: bytes):
    info = orc.column_info(buf)
    out = []
    for c in range(info["n_chunks"]):
        off, ln, r0, rows = orc.chunk_span(buf, c)
        out.append((off, ln, r0, rows, parse_chunk(buf[off:off + ln])))
    return out


def bigint_pack(vals, b: int) -> bytes:
    """Bit-packing as arithmetic: the stream is sum(u_i * 2**(i*b)), little-endian."""
    acc = 0
    for i, v in enumerate(vals):
        acc |= int(v) << (i * b)
    n = (len(vals) * b + 7) // 8
    return acc.to_bytes(n, "little") if n else b""


# ---------------------------------------------------------------------------
# pins
# ---------------------------------------------------------------------------
def pin_bits(orc):
    rng = np.random.default_rng(5)
    xs = [0, 1, 2, 3, 4095, 4096, (1 << 32) - 1, 1 << 32, (1 << 63), (1 << 64) - 1]
    xs += [int(v) for v in rng.integers(0, 1 << 63, 200, dtype=np.int64)]
    for x in xs:
        assert orc.bits(x) == int(x).bit_length(), x


def pin_pack_hand(orc):
    for line in open(os.path.join(GOLDEN, "bitpack_hand.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kv = dict(t.split("=", 1) for t in line.split())
        vals = [int(v) for v in kv["values"].split(",")]
        b = int(kv["b"])
        assert orc.pack(vals, b).hex() == kv["bytes"], line
        assert list(orc.unpack(bytes.fromhex(kv["bytes"]), len(vals), b)) == vals, line


def pin_pack_bruteforce(orc):
    rng = np.random.default_rng(7)
    for b in range(0, 65):
        for n in (0, 1, 2, 3, 7, 8, 9, 31, 33, 64, 70):
            hi = (1 << b) - 1
            vals = [int(v) & hi for v in rng.integers(0, 1 << 63, n, dtype=np.int64) * 2 + rng.integers(0, 2, n)]
            if n >= 2:
                vals[0], vals[-1] = hi, 0
            got = orc.pack(vals, b)
            assert len(got) == (n * b + 7) // 8, (n, b)
            assert got == bigint_pack(vals, b), (n, b)
            if n:
                assert [int(v) for v in orc.unpack(got, n, b)] == vals, (n, b)


def _hand_lines():
    for line in open(os.path.join(GOLDEN, "codecs_hand.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            lhs, rhs = line.split("|")
            scheme, dt, data = lhs.split()
            exp = dict(t.split("=", 1) for t in rhs.split())
            yield scheme, dt, data, exp


def pin_codecs_hand(orc):
    for scheme, dt, data, exp in _hand_lines():
        if dt == "bytes":
            x = np.frombuffer(data.encode(), np.uint8).copy()
        else:
            x = np.array([int(v) for v in data.split(",")], np.int32 if dt == "i32" else np.int64)
        buf = orc.encode(x, O.SCHEMES[scheme], 1 << 20)
        (off, ln, r0, rows, ch), = chunks_of(orc, buf)
        assert ch["scheme"] == O.SCHEMES[scheme] and ch["rows"] == len(x)
        for k, v in exp.items():
            if k.startswith("sec"):
                assert ch["secs"][int(k[3])].hex() == v, (scheme, k, ch["secs"][int(k[3])].hex(), v)
            else:
                assert ch[k] == int(v), (scheme, k, ch[k], v)
        assert np.array_equal(orc.decode(buf), x)


def pin_for_closed_form(orc):
    # 16 chunks of 65,536 values uniform on [0, 4096): 12-bit packing, 98,304 bytes per chunk.
    x = W.uniform_int(1, 0, 0, 1 << 20, 0, 4096).astype(np.int32)
    buf = orc.encode(x, O.FOR_BP, 65536)
    chs = chunks_of(orc, buf)
    assert len(chs) == 16
    total = 0
    for off, ln, r0, rows, ch in chs:
        seg = x[r0:r0 + rows]
        assert ch["bw"] == int(int(seg.max()) - int(seg.min())).bit_length() == 12
        assert ch["ref"] == int(seg.min())
        assert ch["lens"][0] == 98304
        total += ch["lens"][0]
    assert total == 1572864
    assert np.array_equal(orc.decode(buf), x)
    # constant chunk: b = 0, empty payload, every value is the reference
    c = np.full(1000, -77, np.int32)
    (_, _, _, _, ch), = chunks_of(orc, orc.encode(c, O.FOR_BP, 4096))
    assert ch["bw"] == 0 and ch["lens"][0] == 0 and ch["ref"] == -77
    assert np.array_equal(orc.decode(orc.encode(c, O.FOR_BP, 4096)), c)
    # extremes: the full range needs the full width
    for dt, lo, hi, w in ((np.int32, I32_MIN, I32_MAX, 32), (np.int64, I64_MIN, I64_MAX, 64)):
        e = np.array([hi, lo, 0, -1, 1, hi, lo], dt)
        buf = orc.encode(e, O.FOR_BP, 5)
        assert chunks_of(orc, buf)[0][4]["bw"] == w
        assert np.array_equal(orc.decode(buf), e)
    # random widths: b equals the bit length of max - min
    rng = np.random.default_rng(3)
    for w in (1, 5, 17, 31, 33, 47, 62):
        v = rng.integers(-(1 << 62), (1 << 62) - (1 << w), 1).item()
        e = (v + rng.integers(0, 1 << w, 777, dtype=np.int64)).astype(np.int64)
        buf = orc.encode(e, O.FOR_BP, 256)
        for off, ln, r0, rows, ch in chunks_of(orc, buf):
            seg = e[r0:r0 + rows]
            assert ch["bw"] == int(int(seg.max()) - int(seg.min())).bit_length()
            assert ch["lens"][0] == (rows * ch["bw"] + 7) // 8
        assert np.array_equal(orc.decode(buf), e)


def pin_dict(orc):
    x = W.dict_codes(1, 7, 0, 200000)
    buf = orc.encode(x, O.DICT_BP, 65536)
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        seg = x[r0:r0 + rows]
        uniq = np.unique(seg)
        assert ch["n_aux"] == len(uniq)
        assert np.array_equal(np.frombuffer(ch["secs"][0], np.int32), uniq)
        assert ch["bw"] == int(len(uniq) - 1).bit_length()
    assert chunks_of(orc, buf)[0][4]["bw"] == 5  # 25 distinct values
    assert np.array_equal(orc.decode(buf), x)
    for dt in (np.int32, np.int64):
        one = np.full(100, 5, dt)
        b1 = orc.encode(one, O.DICT_BP, 64)
        assert chunks_of(orc, b1)[0][4]["bw"] == 0
        assert np.array_equal(orc.decode(b1), one)
        e = np.array([I64_MAX, I64_MIN, 0, I64_MAX] if dt is np.int64 else [I32_MAX, I32_MIN, 0, I32_MAX], dt)
        assert np.array_equal(orc.decode(orc.encode(e, O.DICT_BP, 3)), e)
    big = np.arange(70000, dtype=np.int32)
    try:
        orc.encode(big, O.DICT_BP, 70000)
    except O.OracleError as err:
        assert err.code == O.EINVAL
    else:
        raise AssertionError("a dictionary above 65,536 entries was accepted")


def pin_delta(orc):
    # arithmetic progression: every difference equals the stride, so b = 0 (DeltaStride, Section 5.3)
    ap = (5 + 7 * np.arange(5000, dtype=np.int64))
    buf = orc.encode(ap, O.DELTA_BP, 1 << 20)
    ch = chunks_of(orc, buf)[0][4]
    assert ch["n_aux"] == 5
    for k in range(5):
        base, min_d, poff, bk = struct.unpack_from("<qqIB", ch["secs"][0], 24 * k)
        assert base == ap[k * 1024] and min_d == 7 and bk == 0
    assert ch["lens"][1] == 0
    assert np.array_equal(orc.decode(buf), ap)
    # sorted keys: round trip; the last value is the base plus the sum of the differences
    keys = W.sorted_keys(2, 300000)
    buf = orc.encode(keys, O.DELTA_BP, 65536)
    dec = orc.decode(buf)
    assert np.array_equal(dec, keys)
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        for k in range(ch["n_aux"]):
            base, min_d, poff, bk = struct.unpack_from("<qqIB", ch["secs"][0], 24 * k)
            seg = keys[r0 + 1024 * k: r0 + min(rows, 1024 * (k + 1))]
            assert base == seg[0]
            assert base + int(np.diff(seg).sum()) == seg[-1]
            if len(seg) > 1:
                d = np.diff(seg)
                assert min_d == d.min() and bk == int(int(d.max()) - int(d.min())).bit_length()
    # wrapping differences at the type's extremes
    for dt, lo, hi in ((np.int32, I32_MIN, I32_MAX), (np.int64, I64_MIN, I64_MAX)):
        e = np.array([hi, lo, 0, -1, hi, hi, lo, lo, 1], dt)
        assert np.array_equal(orc.decode(orc.encode(e, O.DELTA_BP, 4)), e)
    # every int32 array of length <= 3 over a small value set
    vals = [I32_MIN, -1, 0, 1, 2, I32_MAX]
    for n in range(1, 4):
        for idx in np.ndindex(*(len(vals),) * n):
            e = np.array([vals[i] for i in idx], np.int32)
            assert np.array_equal(orc.decode(orc.encode(e, O.DELTA_BP, 2)), e), e


def _check_rle(orc, x, chunk_rows):
    buf = orc.encode(x, O.RLE, chunk_rows)
    total_runs = 0
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        seg = x[r0:r0 + rows]
        vals = np.frombuffer(ch["secs"][0], seg.dtype)
        lens = np.frombuffer(ch["secs"][1], np.uint32)
        assert ch["n_aux"] == len(vals) == len(lens) == np.count_nonzero(np.diff(seg)) + 1
        assert int(lens.sum()) == rows and lens.min() >= 1
        assert np.array_equal(np.repeat(vals, lens), seg)
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        d = np.frombuffer(ch["secs"][2], np.uint32).reshape(-1, 2)
        assert len(d) == (rows + 1023) // 1024
        for t, (fr, skip) in enumerate(d):
            assert starts[fr] + skip == 1024 * t and skip < lens[fr]
        total_runs += len(vals)
    assert np.array_equal(orc.decode(buf), x)
    return buf, total_runs


def pin_rle(orc):
    # Section 5.2.2 distributions: even-X, random[L,R], outlier, mixed
    for kind, a, b in (("even", 2, 0), ("even", 8, 0), ("random", 1, 16), ("outlier", 64, 1024),
                       ("mixed", 4, 32), ("even", 1, 0), ("even", 5000, 0)):
        x = W.rle_distribution(3, kind, 50000, a, b)
        _check_rle(orc, x, 16384)
    # even-8: the count array is 4 bytes per 8 rows = 12.5% of the plain int32 bytes
    x = W.rle_distribution(3, "even", 1 << 16, 8)
    buf, runs = _check_rle(orc, x, 1 << 16)
    ch = chunks_of(orc, buf)[0][4]
    assert ch["lens"][1] * 8 == x.nbytes  # 12.5 %
    # runs are split at chunk boundaries
    y = np.full(3000, 9, np.int64)
    buf, runs = _check_rle(orc, y, 1000)
    assert runs == 3
    _check_rle(orc, W.dates_rle(4, 100000), 32768)


def pin_lz(orc):
    for text in (b"", b"a", b"abc", b"abcd", b"aaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaaa",
                 b"abcabcabcabc" * 50, bytes(range(256)) * 10):
        x = np.frombuffer(text, np.uint8).copy()
        assert np.array_equal(orc.decode(orc.encode(x, O.LZ77, 65536)), x), text[:20]
    # random bytes do not compress: every block is stored raw
    rnd = W.uniform_int(9, 1, 0, 200000, 0, 256).astype(np.uint8)
    buf = orc.encode(rnd, O.LZ77, 65536)
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        assert ch["flags"] & 1 and ch["secs"][0] == rnd[r0:r0 + rows].tobytes()
    assert np.array_equal(orc.decode(buf), rnd)
    # long literal runs need multi-byte varints
    seg = W.uniform_int(9, 2, 0, 3000, 0, 256).astype(np.uint8)
    x = np.concatenate([seg, seg, seg[:500], seg])
    buf = orc.encode(x, O.LZ77, 65536)
    ch = chunks_of(orc, buf)[0][4]
    assert not ch["flags"] & 1 and ch["secs"][0][:2] == bytes([3000 & 0x7F | 0x80, 3000 >> 7])
    assert np.array_equal(orc.decode(buf), x)
    # text round trip, several blocks, a ragged last block
    t, _ = W.text_column(5, 300001)
    buf = orc.encode(t, O.LZ77, 65536)
    assert len(buf) < len(t)
    chs = chunks_of(orc, buf)
    assert len(chs) == 5 and chs[-1][3] == 300001 - 4 * 65536
    assert np.array_equal(orc.decode(buf), t)


def _lz_blob(lengths: bytes, offsets: bytes, lits: bytes, rows: int, ntok: int) -> bytes:
    """A hand-built LZ77 chunk: header, then the lengths, offsets and literal
    streams, each at the next 16-byte boundary."""
    a = 64
    b = (a + len(lengths) + 15) // 16 * 16
    c = (b + len(offsets) + 15) // 16 * 16
    end = (c + len(lits) + 15) // 16 * 16
    blob = bytearray(end)
    struct.pack_into("<IBBBBIIq", blob, 0, 0x4B48435A, O.LZ77, O.BYTES, 0, 0, rows, ntok, 0)
    struct.pack_into("<3I3I", blob, 24, a, b, c, len(lengths), len(offsets), len(lits))
    blob[a:a + len(lengths)] = lengths
    blob[b:b + len(offsets)] = offsets
    blob[c:c + len(lits)] = lits
    return bytes(blob)


def pin_lz_hand_streams(orc):
    # one literal then a back-reference of offset 1: the byte repeats (source overlaps output)
    blob = _lz_blob(bytes([1, 3, 0]), bytes([1, 0]), b"z", 8, 2)
    assert orc.decode_chunk(blob, np.uint8).tobytes() == b"zzzzzzzz"
    # offset 2 over "xy": xyxyxyx
    blob = _lz_blob(bytes([2, 1, 0]), bytes([2, 0]), b"xy", 7, 2)
    assert orc.decode_chunk(blob, np.uint8).tobytes() == b"xyxyxyx"
    # a length may take up to three LEB128 bytes, padded or not: 0x81 0x80 0x00 is 1
    blob = _lz_blob(bytes([0x81, 0x80, 0x00, 0x83, 0x00, 0]), bytes([1, 0]), b"z", 8, 2)
    assert orc.decode_chunk(blob, np.uint8).tobytes() == b"zzzzzzzz"
    # malformed streams are rejected, not decoded
    bad = [
        _lz_blob(bytes([1, 3, 0]), bytes([0, 0]), b"z", 8, 2),      # offset 0
        _lz_blob(bytes([1, 3, 0]), bytes([2, 0]), b"z", 8, 2),      # offset beyond the bytes produced
        _lz_blob(bytes([1, 9, 0]), bytes([1, 0]), b"z", 8, 2),      # match runs past the block
        _lz_blob(bytes([3]), b"", b"z", 3, 1),                      # literals past the literal stream
        _lz_blob(bytes([1, 3, 0, 0]), bytes([1, 0]), b"z", 8, 2),   # unread length bytes
        _lz_blob(bytes([1, 3, 0]), bytes([1, 0, 1, 0]), b"z", 8, 2),  # offsets stream of the wrong size
        _lz_blob(bytes([0x81, 0x80, 0x80, 0x00, 3, 0]), bytes([1, 0]), b"z", 8, 2),  # 4-byte length
        _lz_blob(bytes([1, 3, 0x80]), bytes([1, 0]), b"z", 8, 2),   # last length left open
    ]
    for blob in bad:
        try:
            orc.decode_chunk(blob, np.uint8)
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            raise AssertionError("malformed LZ77 stream accepted")


def pin_chunking(orc):
    x = W.uniform_int(2, 3, 0, 10007, -50, 50).astype(np.int64)
    for scheme in (O.RAW, O.FOR_BP, O.DICT_BP, O.DELTA_BP, O.RLE):
        buf = orc.encode(x, scheme, 1000)
        info = orc.column_info(buf)
        assert info["n_chunks"] == 11 and info["n_rows"] == 10007 and info["total_bytes"] == len(buf)
        prev_end = 64 + 32 * 11
        for c, (off, ln, r0, rows, ch) in enumerate(chunks_of(orc, buf)):
            assert off == prev_end and off % 16 == 0 and ln % 16 == 0
            assert r0 == 1000 * c and rows == min(1000, 10007 - r0)
            assert all(o % 16 == 0 for o, l in zip(ch["offs"], ch["lens"]) if o or l)
            assert np.array_equal(orc.decode_chunk(buf[off:off + ln], np.int64), x[r0:r0 + rows])
            prev_end = off + ln
        assert np.array_equal(orc.decode(buf), x)
    empty = orc.encode(np.zeros(0, np.int32), O.FOR_BP, 1000)
    assert orc.column_info(empty)["n_chunks"] == 0 and len(orc.decode(empty)) == 0


def pin_rejects_corrupt(orc):
    x = W.uniform_int(2, 3, 0, 5000, 0, 1000).astype(np.int32)
    for scheme in (O.FOR_BP, O.DELTA_BP, O.RLE):
        buf = bytearray(orc.encode(x, scheme, 5000))
        off, ln, r0, rows, ch = chunks_of(orc, bytes(buf))[0]
        bad = bytearray(buf)
        bad[off] ^= 0xFF  # chunk magic
        try:
            orc.decode(bytes(bad))
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            raise AssertionError("bad magic accepted")
    # RLE counts that do not add up to the rows
    buf = bytearray(orc.encode(x, O.RLE, 5000))
    off, ln, r0, rows, ch = chunks_of(orc, bytes(buf))[0]
    lo = off + ch["offs"][1]
    struct.pack_into("<I", buf, lo, struct.unpack_from("<I", buf, lo)[0] + 1)
    try:
        orc.decode(bytes(buf))
    except O.OracleError as err:
        assert err.code == O.ECORRUPT
    else:
        raise AssertionError("RLE count mismatch accepted")


def pin_strings(orc):
    t, o = W.text_column(6, 200000)
    buf = orc.encode_strings(t, o)
    t2, o2 = orc.decode_strings(buf)
    assert np.array_equal(t2, t) and np.array_equal(o2, o)
    assert o[0] == 0 and o[-1] == len(t) and np.all(np.diff(o) > 0)



# ---- Float2Int (Section 2.1 "Float2Int"; Table 2 pairs it with bit-packing) ----

def _f2i_blob(e: int, b: int, ref: int, packed: bytes, pos, vals, rows: int) -> bytes:
    """A hand-built Float2Int chunk: header (exponent e in byte 48), then the
    packed integers, the exception rows and the exception bit patterns."""
    ex_pos = b"".join(struct.pack("<I", p) for p in pos)
    ex_val = b"".join(struct.pack("<d", v) for v in vals)
    a = 64
    bb = (a + len(packed) + 15) // 16 * 16
    c = (bb + len(ex_pos) + 15) // 16 * 16
    end = (c + len(ex_val) + 15) // 16 * 16
    blob = bytearray(max(end, 64))
    struct.pack_into("<IBBBBIIq", blob, 0, 0x4B48435A, O.FLOAT2INT, O.F64, b, 0, rows, len(pos), ref)
    struct.pack_into("<3I3I", blob, 24, a, bb, c, len(packed), len(ex_pos), len(ex_val))
    blob[48] = e
    blob[a:a + len(packed)] = packed
    blob[bb:bb + len(ex_pos)] = ex_pos
    blob[c:c + len(ex_val)] = ex_val
    return bytes(blob)


def _same_bits(x, y) -> bool:
    return np.array_equal(np.asarray(x, np.float64).view(np.uint64), np.asarray(y, np.float64).view(np.uint64))


def pin_f2i_hand_example(orc):
    # 1.25, 3.5, 10, 0.75 are the integers 125, 350, 1000, 75 at e = 2 (at e = 1,
    # 1.25 * 10 = 12.5 rounds to 12 and 1.2 != 1.25): reference 75, u = 50,
    # 275, 925, 0, b = bits(925) = 10, packed LSB-first
    x = np.array([1.25, 3.5, 10.0, 0.75])
    buf = orc.encode(x, O.FLOAT2INT, 1000)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    blob = buf[off:off + ln]
    assert (ch["bw"], ch["ref"], ch["n_aux"], blob[48]) == (10, 75, 0, 2)
    assert ch["secs"][0] == bigint_pack([50, 275, 925, 0], 10) == bytes.fromhex("324cd43900")
    assert _same_bits(orc.decode(buf), x)


def pin_f2i_value_is_the_nearest_double(orc):
    # the decoded value of integer d at exponent e is the double nearest to
    # d / 10^e: Python's Fraction -> float conversion rounds correctly
    from fractions import Fraction
    rng = np.random.default_rng(5)
    for e in range(0, 19):
        for scale in (10, 10**6, 2**40, 2**53 - 1):
            d = [int(v) for v in rng.integers(-scale, scale, 200, dtype=np.int64)] + [scale, -scale, 0, 1, -1]
            ref = min(d)
            u = [v - ref for v in d]
            b = max(u).bit_length()
            blob = _f2i_blob(e, b, ref, bigint_pack(u, b), [], [], len(d))
            got = orc.decode_chunk(blob, np.float64)
            want = np.array([float(Fraction(v, 10 ** e)) for v in d])
            assert _same_bits(got, want), (e, scale)


def pin_f2i_decimal_prices(orc):
    # prices with two decimals (the double nearest cents / 100) all come back
    # from their integer cents at e = 2: no exceptions, reference = the
    # chunk's smallest cents, width = bits(max - min)
    rng = np.random.default_rng(6)
    cents = np.round(np.exp(rng.normal(11.5, 1.0, 30000))).astype(np.int64)
    cents[::7] += 1                                   # make sure odd cents occur
    x = cents / 100.0
    buf = orc.encode(x, O.FLOAT2INT, 10000)
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        c = cents[r0:r0 + rows]
        assert buf[off + 48] == 2 and ch["n_aux"] == 0
        assert ch["ref"] == c.min() and ch["bw"] == int(c.max() - c.min()).bit_length()
    assert _same_bits(orc.decode(buf), x)
    # integer-valued doubles need no scaling
    y = np.arange(-500, 500, dtype=np.float64) * 3
    buf = orc.encode(y, O.FLOAT2INT, 4096)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    assert buf[off + 48] == 0 and ch["n_aux"] == 0 and ch["ref"] == -1500 and ch["bw"] == 12
    assert _same_bits(orc.decode(buf), y)


def pin_f2i_exceptions(orc):
    # values that are not decimals of at most 18 digits after the point, or
    # whose integer would reach 2^53, are kept bit for bit as exceptions
    sp = np.array([np.nan, np.inf, -np.inf, -0.0, 0.0, 1e300, 5e-324, 0.1 + 0.2, 1 / 3, 2.0 ** 60, -7.5])
    buf = orc.encode(sp, O.FLOAT2INT, 1000)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    # only 0.0 and -7.5 fit (at e = 1, the smallest exponent that takes -7.5)
    assert buf[off + 48] == 1 and ch["n_aux"] == 9
    assert list(struct.unpack_from("<9I", ch["secs"][1])) == [0, 1, 2, 3, 5, 6, 7, 8, 9]
    assert _same_bits(orc.decode(buf), sp)
    # a hand-built chunk: rows 1 and 3 are replaced by the stored bits
    blob = _f2i_blob(0, 2, 5, bigint_pack([0, 1, 2, 3], 2), [1, 3], [-0.0, 0.5], 4)
    assert _same_bits(orc.decode_chunk(blob, np.float64), [5.0, -0.0, 7.0, 0.5])
    # malformed: rows out of order or out of range, exponent above 18, sizes
    bad = [
        _f2i_blob(0, 2, 5, bigint_pack([0, 1, 2, 3], 2), [3, 1], [1.0, 2.0], 4),
        _f2i_blob(0, 2, 5, bigint_pack([0, 1, 2, 3], 2), [4], [1.0], 4),
        _f2i_blob(19, 2, 5, bigint_pack([0, 1, 2, 3], 2), [], [], 4),
        _f2i_blob(0, 3, 5, bigint_pack([0, 1, 2, 3], 2), [], [], 4),
        # an integer beyond 2^53 (the encoder stores |d| <= 2^53 only), either sign
        _f2i_blob(2, 1, 2**53, bigint_pack([0, 1], 1), [], [], 2),
        _f2i_blob(2, 1, -2**53 - 1, bigint_pack([1, 0], 1), [], [], 2),
    ]
    # the bounds themselves are valid: +-2^53 / 10^2
    ok = orc.decode_chunk(_f2i_blob(2, 55, -2**53, bigint_pack([0, 2**54], 55), [], [], 2), np.float64)
    assert _same_bits(ok, [float(-2**53) / 100, float(2**53) / 100])
    for blob in bad:
        try:
            orc.decode_chunk(blob, np.float64)
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            raise AssertionError("malformed Float2Int chunk accepted")


# ---- string dictionary + bit-packing (Section 2.1 dictionary encoding over the
# ---- words of a text column, as Section 5.3.1 does for the comment column) ----

def _plain_tokens(chunk: bytes, starts: set) -> list:
    """Tokens of one chunk by the format's rule, written with Python slicing:
    cut after every space, before every row start, every 64 bytes."""
    toks, cur = [], b""
    for i, c in enumerate(chunk):
        if cur and (i in starts or len(cur) == 64):
            toks.append(cur)
            cur = b""
        cur += bytes([c])
        if c == 0x20:
            toks.append(cur)
            cur = b""
    if cur:
        toks.append(cur)
    return toks


def _plain_strdict_chunk(chunk: bytes, starts: set):
    toks = _plain_tokens(chunk, starts)
    d = sorted(set(toks))
    if len(d) > 65536:
        toks = [bytes([c]) for c in chunk]
        d = sorted(set(toks))
    rank = {t: k for k, t in enumerate(d)}
    offs = np.cumsum([0] + [len(t) for t in d]).tolist()
    tiles, pos = [], 0
    for i, t in enumerate(toks):
        if i % 1024 == 0:
            tiles.append(pos)
        pos += len(t)
    b = (len(d) - 1).bit_length()
    return d, [rank[t] for t in toks], offs, tiles, b


def pin_strdict_hand_example(orc):
    # rows "ab cd" and "ab": tokens "ab ", "cd" | "ab"; sorted dictionary
    # "ab" < "ab " < "cd"; codes 1, 2, 0 at 2 bits = 0b00_10_01
    t = np.frombuffer(b"ab cdab", np.uint8).copy()
    buf = orc.encode_strdict(t, np.array([0, 5, 7], np.int32), 65536)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    assert (ch["scheme"], ch["dtype"], ch["bw"], ch["rows"], ch["n_aux"], ch["ref"]) == (7, 2, 2, 7, 3, 3)
    assert ch["secs"][0] == struct.pack("<5I", 0, 2, 5, 7, 0)
    assert ch["secs"][1] == b"abab cd"
    assert ch["secs"][2] == bytes([0x09])
    assert orc.decode(buf).tobytes() == b"ab cdab"


def pin_strdict_matches_the_plain_tokenizer(orc):
    rng = np.random.default_rng(17)
    words = [b"a", b"bb", b"ccc", b"the", b"x" * 70, b"", b"  ", b"q r"]
    for trial in range(6):
        rows = [b" ".join(words[k] for k in rng.integers(0, len(words), rng.integers(0, 6)))
                for _ in range(rng.integers(1, 400))]
        t = np.frombuffer(b"".join(rows) or b"", np.uint8).copy()
        o = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
        if len(t) == 0:
            continue
        chunk = 65536 if trial % 2 else 1 << 16
        buf = orc.encode_strdict(t, o, chunk)
        data = t.tobytes()
        for off, ln, r0, rows_c, ch in chunks_of(orc, buf):
            piece = data[r0:r0 + rows_c]
            starts = {int(x) - r0 for x in o if r0 < x < r0 + rows_c}
            d, codes, offs, tiles, b = _plain_strdict_chunk(piece, starts)
            assert ch["n_aux"] == len(d) and ch["ref"] == len(codes) and ch["bw"] == b
            assert ch["secs"][1] == b"".join(d)
            assert ch["secs"][0] == struct.pack(f"<{len(offs) + len(tiles)}I", *offs, *tiles)
            assert ch["secs"][2] == bigint_pack(codes, b)
        assert orc.decode(buf).tobytes() == data


def pin_strdict_round_trip_and_byte_tokens(orc):
    t, o = W.text_column(9, 300000)
    buf = orc.encode_strings(t, o, 131072, scheme=O.STRDICT)
    t2, o2 = orc.decode_strings(buf)
    assert np.array_equal(t2, t) and np.array_equal(o2, o)
    # 70,000 distinct five-byte tokens in one chunk: above 65,536, so every byte is a token
    k = np.arange(70000)
    words = np.stack([97 + k % 26, 97 + k // 26 % 26, 97 + k // 676 % 26, 97 + k // 17576 % 26,
                      np.full_like(k, 32)], 1).astype(np.uint8)
    data = words.reshape(-1)
    buf = orc.encode_strdict(data, np.array([0, len(data)], np.int32), 1 << 19)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    assert ch["ref"] == len(data) and ch["n_aux"] == len(np.unique(data)) and ch["bw"] == 5
    assert np.array_equal(orc.decode(buf), data)


def pin_strdict_rejects_corrupt(orc):
    t = np.frombuffer(b"ab cdab", np.uint8).copy()
    buf = orc.encode_strdict(t, np.array([0, 5, 7], np.int32), 65536)
    (off, ln, r0, rows, ch), = chunks_of(orc, buf)
    blob = bytearray(buf[off:off + ln])
    o0, o1, o2 = ch["offs"]
    bad = []
    b1 = bytearray(blob); b1[o2] = 0x0D; bad.append(b1)                             # code 3 >= 3 entries
    b2 = bytearray(blob); struct.pack_into("<I", b2, o0 + 16, 1); bad.append(b2)    # first tile starts at 1
    b3 = bytearray(blob); struct.pack_into("<I", b3, o0 + 4, 5); bad.append(b3)     # entries not increasing
    b4 = bytearray(blob); b4[6] = 3; bad.append(b4)                                 # width is not bits(ndict - 1)
    for bb in bad:
        try:
            orc.decode_chunk(bytes(bb), np.uint8)
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            raise AssertionError("malformed string-dictionary chunk accepted")


# ---- dictionary + ANS (Section 2.1 entropy-based algorithms; Section 3.1 takes
# ---- ANS decode as the Non-Parallel example; the coder is Duda's rANS) ----

def _ans_parts(orc, x, chunk_rows):
    """(frequencies, stream starts, streams, state words) of every chunk."""
    buf = orc.encode(x, O.ANS, chunk_rows)
    out = []
    for off, ln, r0, rows, ch in chunks_of(orc, buf):
        nd, K = ch["n_aux"], ch["ref"]
        fb = (2 * nd + 3) // 4 * 4
        f = list(struct.unpack_from(f"<{nd}H", ch["secs"][1]))
        starts = list(struct.unpack_from(f"<{K + 1}I", ch["secs"][1], fb))
        out.append((ch, f, starts))
    return buf, out


def pin_ans_frequencies(orc):
    # f_s = max(1, floor(count * 4096 / n)); a shortfall goes to the most
    # frequent symbol (the first on a tie), an excess leaves the largest f_s
    cases = [
        (np.array([5, 7, 7, 9], np.int32), [1024, 2048, 1024]),
        (np.array([1, 2, 3], np.int32), [1366, 1365, 1365]),
        (np.array([0] * 9999 + [1], np.int64), [4095, 1]),
        (np.arange(256, dtype=np.int32), [16] * 256),
        (np.full(777, -3, np.int64), [4096]),
        # 255 symbols once and one symbol 4000 times: floor gives 0 -> 1 for the
        # rare ones (255), and floor(4000 * 4096 / 4255) = 3850 for the common one:
        # 4105 in all, 9 too many, all taken from the largest
        (np.array(list(range(255)) + [1000] * 4000, np.int32), [1] * 255 + [3841]),
    ]
    for x, want in cases:
        _, parts = _ans_parts(orc, x, 1 << 20)
        (ch, f, starts), = parts
        assert f == want and sum(f) == 4096 and ch["bw"] == 12, (f[:4], want[:4])
        assert np.array_equal(orc.decode(orc.encode(x, O.ANS, 1 << 20)), x)


def pin_ans_size_is_the_information(orc):
    # Each coding step multiplies the state by about M / f_s, so a stream's
    # emitted bits plus log2(final state / L) equal sum(log2(4096 / f_s)) over
    # its rows, up to 2^-11 relative per step; 16 equal symbols cost exactly
    # 4 bits each, so every 512-row stream is 4 + 256 bytes.
    rng = np.random.default_rng(21)
    x = np.repeat(np.arange(16, dtype=np.int32), 256)
    rng.shuffle(x)
    _, ((ch, f, starts),) = _ans_parts(orc, x, 4096)
    assert f == [256] * 16 and starts == [260 * k for k in range(9)] and ch["lens"][2] == 2080
    for x in (rng.choice([65, 78, 82], 4096, p=[0.25, 0.5, 0.25]).astype(np.int32),
              (rng.geometric(0.2, 4096) % 150).astype(np.int64)):
        _, ((ch, f, starts),) = _ans_parts(orc, x, 4096)
        vals = np.unique(x)
        s2 = ch["secs"][2]
        for k in range(len(starts) - 1):
            rows = x[512 * k:512 * (k + 1)]
            need = sum(np.log2(4096 / f[np.searchsorted(vals, v)]) for v in rows)
            q = s2[starts[k]:starts[k + 1]]
            got = 8 * (len(q) - 4) + np.log2(struct.unpack_from("<I", q)[0]) - 23
            assert abs(got - need) <= 1 + len(rows) * 2.0 ** -10, (k, got, need)


def pin_ans_round_trip_and_streams(orc):
    rng = np.random.default_rng(22)
    cases = [
        rng.choice([65, 78, 82], 100001, p=[0.25, 0.5, 0.25]).astype(np.int32),   # ragged, several streams
        rng.integers(I64_MIN, I64_MAX, 256, dtype=np.int64)[rng.integers(0, 256, 9000)],
        np.full(5000, 7, np.int64),
        np.array([I32_MIN, I32_MAX] * 3000, np.int32),
    ]
    for x in cases:
        buf, parts = _ans_parts(orc, x, 65536)
        assert np.array_equal(orc.decode(buf), x)
        for ch, f, starts in parts:
            K = (ch["rows"] + 511) // 512
            assert ch["b48"] == 9                          # 512 rows per stream unless named
            assert ch["ref"] == K and len(starts) == K + 1 and starts[0] == 0
            assert starts[-1] == ch["lens"][2] and all(b - a >= 4 for a, b in zip(starts, starts[1:]))
    try:
        orc.encode(np.arange(257, dtype=np.int32), O.ANS, 65536)
    except O.OracleError as err:
        assert err.code == O.EINVAL
    else:
        raise AssertionError("257 distinct values accepted by the ANS encoder")


def pin_ans_stream_length(orc):
    # Section 5.2.3 trades ratio for throughput through the ANS chunk size;
    # here each chunk names its rows per stream L = 2^k (header byte 48 = k,
    # 5 <= k <= 12) and holds K = ceil(rows / L) streams
    rng = np.random.default_rng(24)
    x = np.repeat(np.arange(16, dtype=np.int32), 640)
    rng.shuffle(x)                                          # 10,240 rows, 16 equal symbols: 4 bits a row
    sizes = []
    for k in range(5, 13):
        L = 1 << k
        buf = orc.encode(x, O.ANS, 1 << 20, ans_stream_rows=L)
        (off, ln, r0, rows, ch), = chunks_of(orc, buf)
        K = -(-len(x) // L)
        nd = ch["n_aux"]
        starts = list(struct.unpack_from(f"<{K + 1}I", ch["secs"][1], (2 * nd + 3) // 4 * 4))
        assert ch["b48"] == k and ch["ref"] == K and len(ch["secs"][1]) == 32 + 4 * (K + 1)
        # each stream: the 4-byte state and exactly half a byte per row
        lens = [(min(L, len(x) - L * j) + 1) // 2 + 4 for j in range(K)]
        assert [b - a for a, b in zip(starts, starts[1:])] == lens, k
        assert np.array_equal(orc.decode(buf), x)
        sizes.append(len(buf))
    assert sizes == sorted(sizes, reverse=True)             # fewer streams, fewer bytes
    for L in (16, 48, 8192):
        try:
            orc.encode(x, O.ANS, 1 << 20, ans_stream_rows=L)
        except O.OracleError as err:
            assert err.code == O.EINVAL
        else:
            raise AssertionError(f"{L} rows per ANS stream accepted")
    # a chunk whose length byte disagrees with its streams is malformed
    buf = orc.encode(x[:3000], O.ANS, 1 << 20, ans_stream_rows=256)
    off, ln, _, _ = orc.chunk_span(buf, 0)
    for k in (4, 13, 7, 9):
        bb = bytearray(buf[off:off + ln])
        bb[48] = k
        try:
            orc.decode_chunk(bytes(bb), np.int32)
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            raise AssertionError(f"ANS chunk with stream length byte {k} accepted")


def pin_ans_rejects_corrupt(orc):
    x = np.random.default_rng(23).choice([1, 2, 3, 4], 9000, p=[0.4, 0.3, 0.2, 0.1]).astype(np.int32)
    buf, ((ch, f, starts),) = _ans_parts(orc, x, 65536)
    off = orc.chunk_span(buf, 0)[0]
    blob = bytes(buf[off:off + orc.chunk_span(buf, 0)[1]])
    o1, o2 = ch["offs"][1], ch["offs"][2]
    bad = []
    b1 = bytearray(blob); struct.pack_into("<H", b1, o1, f[0] + 1); bad.append(b1)         # sum above 4096
    b2 = bytearray(blob); struct.pack_into("<I", b2, o1 + 8 + 4, starts[1] + 1); bad.append(b2)  # stream start
    b3 = bytearray(blob); b3[o2 + 4] ^= 0x40; bad.append(b3)                                # a stream byte
    b4 = bytearray(blob); b4[6] = 11; bad.append(b4)                                       # scale bits
    for bb in bad:
        try:
            got = orc.decode_chunk(bytes(bb), np.int32)
        except O.OracleError as err:
            assert err.code == O.ECORRUPT
        else:
            assert not np.array_equal(got, x), "corrupt ANS chunk decoded to the column"
            raise AssertionError("malformed ANS chunk accepted")


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
