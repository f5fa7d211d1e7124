"""Host-side checks of libzf.so (no GPU needed): the ABI is exported, the
library's encoder writes the oracle's bytes for every canonical scheme, LZ77
streams cross-decode, and malformed containers are rejected."""
import os
import re
import struct

import numpy as np
import pytest

import oracle
import zf_workloads as W
from oracle_pins import chunks_of, parse_chunk

zf = pytest.importorskip("paper_2602_08190_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def lib_encode(x, scheme, chunk_rows=65536, offsets=None, offsets_scheme=-1):
    col = zf.Column(x, offsets)
    p = zf.zf_plan(None, col, scheme=scheme, chunk_rows=chunk_rows, offsets_scheme=offsets_scheme)
    c = zf.zf_compress_host(p, col)
    try:
        return zf.zf_compressed_bytes(c)
    finally:
        zf.zf_compressed_free(c)


def test_exports_every_declared_symbol():
    hdr = open(os.path.join(ROOT, "include", "zf.h")).read()
    declared = set(re.findall(r"^\s*(?:zf_status|const char\*)\s+(zf_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    import ctypes
    lib = ctypes.CDLL(zf.LIB_PATH)
    missing = [s for s in sorted(declared) if not hasattr(lib, s)]
    assert not missing, missing
    assert declared <= set(zf.EXPORTED) | declared


def _cases():
    I32, I64 = np.int32, np.int64
    rng = np.random.default_rng(11)
    yield "c1_uniform12", W.uniform_int(1, 0, 0, 300000, 0, 4096).astype(I32), 65536
    yield "keys", W.sorted_keys(3, 250000), 1 << 17
    yield "dates", W.dates_rle(3, 250000), 1 << 17
    yield "dict25", W.dict_codes(3, 7, 0, 100000), 32768
    yield "lognormal", W.lognormal_cents(3, 9, 0, 100000), 32768
    yield "i32_extremes", np.array([2**31 - 1, -2**31, 0, -1, 5] * 999, I32), 1024
    yield "i64_extremes", np.array([2**63 - 1, -2**63, 0, -1, 5] * 999, I64), 2048
    yield "ragged", rng.integers(-1000, 1000, 12345).astype(I64), 4096
    yield "constant", np.full(5000, 42, I32), 1024
    yield "one_row", np.array([7], I64), 1024
    yield "outlier_runs", W.rle_distribution(2, "outlier", 70000, 64, 1024), 16384
    yield "mixed_runs", W.rle_distribution(2, "mixed", 70000, 4, 32), 16384


@pytest.mark.parametrize("scheme", ["raw", "for_bp", "dict_bp", "delta_bp", "rle"])
@pytest.mark.parametrize("case", list(_cases()), ids=lambda c: c[0])
def test_encoder_bytes_equal_oracle(scheme, case):
    name, x, cr = case
    s = oracle.SCHEMES[scheme]
    try:
        ob = oracle.encode(x, s, cr)
    except oracle.OracleError:
        with pytest.raises(zf.ZfError):
            lib_encode(x, s, cr)
        return
    lb = lib_encode(x, s, cr)
    assert len(lb) == len(ob)
    assert lb == ob


def test_dictionary_limit_rejected():
    with pytest.raises(zf.ZfError) as e:
        lib_encode(np.arange(70000, dtype=np.int32), zf.ZF_DICT_BP, 70656)
    assert e.value.status == zf.ZF_EINVAL


def test_lz77_cross_decode():
    t, o = W.text_column(8, 400000)
    lb = lib_encode(t, zf.ZF_LZ77, offsets=o)
    t2, o2 = oracle.decode_strings(lb)
    assert np.array_equal(t2, t) and np.array_equal(o2, o)
    # the library compresses at least as well as the oracle's simpler encoder here
    assert len(lb) <= len(oracle.encode_strings(t, o))
    # oracle-encoded strings pass the library's structural validation
    c = zf.zf_compressed_from_bytes(oracle.encode_strings(t, o))
    raw, comp, n = zf.zf_compressed_info(c)
    assert raw == len(t) + 4 * len(o)
    zf.zf_compressed_free(c)


def test_lz77_random_bytes_stored_raw():
    r = W.uniform_int(5, 5, 0, 200000, 0, 256).astype(np.uint8)
    o = np.array([0, 100000, 200000], np.int32)
    lb = lib_encode(r, zf.ZF_LZ77, offsets=o)
    info = oracle.column_info(lb)
    for c in range(info["n_chunks"]):
        off, ln, r0, rows = oracle.chunk_span(lb, c)
        assert lb[off + 7] & 1
    t2, o2 = oracle.decode_strings(lb)
    assert np.array_equal(t2, r)


def test_from_bytes_round_trip_and_rejects_corruption():
    x = W.dates_rle(4, 50000)
    b = oracle.encode(x, oracle.RLE, 16384)
    c = zf.zf_compressed_from_bytes(b)
    assert zf.zf_compressed_bytes(c) == b
    zf.zf_compressed_free(c)
    bad_cases = []
    bb = bytearray(b); bb[0] ^= 1; bad_cases.append(bb)                      # column magic
    bb = bytearray(b); struct.pack_into("<Q", bb, 64, 80); bad_cases.append(bb)  # directory offset
    off = oracle.chunk_span(b, 1)[0]
    bb = bytearray(b); bb[off] ^= 1; bad_cases.append(bb)                    # chunk magic
    bb = bytearray(b); struct.pack_into("<I", bb, off + 36, 1 << 30); bad_cases.append(bb)  # section length
    bad_cases.append(bytearray(b[:-16]))                                     # truncated
    one = oracle.encode(x[:10000], oracle.RLE, 16384)                        # one chunk: only the bound fails
    bb = bytearray(one); struct.pack_into("<I", bb, 12, 1 << 31); bad_cases.append(bb)  # chunk_rows above 2^30
    for bb in bad_cases:
        with pytest.raises(zf.ZfError) as e:
            zf.zf_compressed_from_bytes(bytes(bb))
        assert e.value.status == zf.ZF_ECORRUPT


def test_plan_heuristic_picks_the_obvious_scheme():
    def pick(x):
        return zf.zf_plan(None, zf.Column(x), scheme=-1, chunk_rows=65536).scheme
    assert pick(W.sorted_keys(1, 200000)) == zf.ZF_DELTA_BP
    assert pick(W.rle_distribution(1, "even", 200000, 64)) == zf.ZF_RLE
    assert pick(W.uniform_int(1, 2, 0, 200000, 0, 4096).astype(np.int32)) == zf.ZF_FOR_BP
    assert pick(W.dict_codes(1, 3, 0, 200000)) == zf.ZF_DICT_BP
    with pytest.raises(zf.ZfError):
        zf.zf_plan(None, zf.Column(np.zeros(10, np.int32)), scheme=zf.ZF_FOR_BP, chunk_rows=1000)


def _float_cases():
    rng = np.random.default_rng(31)
    prices = W.decimal_prices(3, 5, 0, 100_000)
    mixed = prices[:20_000].copy()
    mixed[::997] = np.nan
    mixed[5::1999] = np.inf
    mixed[7::2999] = -0.0
    mixed[11::3001] = 1.0 / 3.0
    yield "prices_2dp", prices, 32768
    yield "prices_3dp", W.decimal_prices(4, 5, 0, 50_000, 3), 16384
    yield "integers", rng.integers(-10**12, 10**12, 30_000).astype(np.float64), 8192
    yield "mixed_exceptions", mixed, 4096
    yield "random_doubles", rng.standard_normal(9_000), 4096
    yield "one_row", np.array([12.5]), 1024
    yield "empty", np.zeros(0, np.float64), 1024


FLOAT_CASES = list(_float_cases())


@pytest.mark.parametrize("scheme", ["raw", "float2int"])
@pytest.mark.parametrize("case", FLOAT_CASES, ids=lambda c: c[0])
def test_float2int_encoder_bytes_equal_oracle(scheme, case):
    """Float2Int is canonical (exponent with the fewest exceptions, smallest
    on a tie): the library writes the oracle's bytes, and both decode to the
    column bit for bit."""
    name, x, cr = case
    s = oracle.SCHEMES[scheme]
    ob = oracle.encode(x, s, cr)
    lb = lib_encode(x, s, cr)
    assert lb == ob
    assert np.array_equal(oracle.decode(lb).view(np.uint64), x.view(np.uint64))


def test_float2int_plan_and_validation():
    x = W.decimal_prices(1, 5, 0, 5000)
    p = zf.zf_plan(None, zf.Column(x))
    assert p.scheme == zf.ZF_FLOAT2INT
    with pytest.raises(zf.ZfError):               # integer schemes do not take doubles
        lib_encode(x, zf.ZF_FOR_BP, 1024)
    b = lib_encode(np.array([1.5, np.nan, 2.25, np.inf]), zf.ZF_FLOAT2INT, 1024)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    assert ch["n_aux"] == 2
    # exception rows out of order are rejected by the host check
    bad = bytearray(b)
    p1 = off + ch["offs"][1]
    bad[p1:p1 + 8] = struct.pack("<II", 3, 1)
    with pytest.raises(zf.ZfError) as e:
        zf.zf_compressed_from_bytes(bytes(bad))
    assert e.value.status == zf.ZF_ECORRUPT


def test_column_rejects_unsupported_dtypes():
    with pytest.raises(TypeError):
        zf.Column(np.zeros(8, np.int16))
    with pytest.raises(TypeError):
        zf.Column(np.zeros(8, np.int32), np.array([0, 8], np.int32))   # string bytes must be uint8
    assert zf.Column(np.zeros(8, np.float64)).c.dtype == zf.ZF_F64


def test_strdict_bytes_equal_the_oracle():
    """String dictionary + bit-packing: the library's encoder writes the same
    bytes as the oracle (the encoding is canonical), for several chunk sizes."""
    cases = [(W.text_column(3, 1000003), 1 << 20), (W.text_column(4, 200000), 65536),
             ((np.frombuffer(b"ab cdab", np.uint8).copy(), np.array([0, 5, 7], np.int32)), 65536)]
    rng = np.random.default_rng(3)
    raw = rng.integers(0, 256, 150000).astype(np.uint8)              # few spaces: long tokens, byte-heavy
    cases.append(((raw, np.array([0, 70000, 70000, 150000], np.int32)), 131072))
    for (t, o), cb in cases:
        col = zf.Column(t, o)
        h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_STRDICT, chunk_rows=cb), col)
        try:
            lb = zf.zf_compressed_bytes(h)
            assert lb == oracle.encode_strings(t, o, cb, scheme=oracle.STRDICT)
            t2, o2 = oracle.decode_strings(lb)
            assert np.array_equal(t2, t) and np.array_equal(o2, o)
        finally:
            zf.zf_compressed_free(h)


def test_strdict_plan_and_host_checks():
    t, o = W.text_column(5, 300000)
    col = zf.Column(t, o)
    assert zf.zf_plan(None, col, scheme=zf.ZF_STRDICT).chunk_rows == 4 << 20
    for cb in (65536 + 1024, 1 << 27):
        with pytest.raises(zf.ZfError):
            zf.zf_plan(None, col, scheme=zf.ZF_STRDICT, chunk_rows=cb)
    b = oracle.encode_strings(t, o, 131072, scheme=oracle.STRDICT)
    off = oracle.chunk_span(b, 0)[0]
    ch = parse_chunk(b[off:off + 64])
    nd = ch["n_aux"]
    bad_cases = []
    bb = bytearray(b); struct.pack_into("<I", bb, off + ch["offs"][0] + 4, 0); bad_cases.append(bb)  # empty entry
    bb = bytearray(b); struct.pack_into("<I", bb, off + ch["offs"][0] + 4 * (nd + 1), 3); bad_cases.append(bb)  # tile 0 at 3
    bb = bytearray(b); bb[off + 6] += 1; bad_cases.append(bb)                                        # code width
    bb = bytearray(b); struct.pack_into("<I", bb, 12, 65536 + 1024); bad_cases.append(bb)          # chunk bytes
    for bb in bad_cases:
        with pytest.raises(zf.ZfError) as e:
            zf.zf_compressed_from_bytes(bytes(bb))
        assert e.value.status == zf.ZF_ECORRUPT


def _ans_cases():
    rng = np.random.default_rng(1)
    return [rng.choice([65, 78, 82], 100001, p=[0.25, 0.5, 0.25]).astype(np.int32),
            rng.integers(I64_LO, I64_HI, 256, dtype=np.int64)[rng.integers(0, 256, 9000)],
            np.full(5000, 7, np.int64), np.array([-2**31, 2**31 - 1] * 3000, np.int32),
            (rng.geometric(0.05, 300000) % 256).astype(np.int32),
            np.array(list(range(255)) + [1000] * 4000, np.int32)]


I64_LO, I64_HI = -(1 << 63), (1 << 63) - 1


def test_ans_bytes_equal_the_oracle():
    """Dictionary + ANS: the library's encoder writes the oracle's bytes
    (canonical frequencies, streams of 512 rows)."""
    for x in _ans_cases():
        for cr in (1024, 65536, 1 << 20):
            col = zf.Column(x)
            h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS, chunk_rows=cr), col)
            try:
                lb = zf.zf_compressed_bytes(h)
                assert lb == oracle.encode(x, oracle.ANS, cr), (len(x), cr)
            finally:
                zf.zf_compressed_free(h)
    col = zf.Column(np.arange(300, dtype=np.int32))                     # 300 values in one chunk
    with pytest.raises(zf.ZfError) as e:
        zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS), col)
    assert e.value.status == zf.ZF_EINVAL


@pytest.mark.parametrize("stream_rows", [32, 64, 128, 256, 1024, 2048, 4096])
def test_ans_stream_lengths_bytes_equal_the_oracle(stream_rows):
    """Every stream length (header byte 48): the library's bytes equal the
    oracle's; a length that is not a power of two in 32..4096 is refused."""
    for x in _ans_cases()[:3]:
        for cr in (1024, 65536):
            col = zf.Column(x)
            h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS, chunk_rows=cr,
                                               ans_stream_rows=stream_rows), col)
            try:
                assert zf.zf_compressed_bytes(h) == oracle.encode(x, oracle.ANS, cr, ans_stream_rows=stream_rows)
            finally:
                zf.zf_compressed_free(h)
    col = zf.Column(_ans_cases()[0])
    for bad in (16, 48, 8192):
        with pytest.raises(zf.ZfError) as e:
            zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS, ans_stream_rows=bad), col)
        assert e.value.status == zf.ZF_EINVAL


def test_ans_host_checks():
    x = _ans_cases()[0]
    b = oracle.encode(x, oracle.ANS, 65536)
    off = oracle.chunk_span(b, 0)[0]
    ch = parse_chunk(b[off:off + 64])
    o1 = off + ch["offs"][1]
    bad = []
    bb = bytearray(b); struct.pack_into("<H", bb, o1, 0); bad.append(bb)                     # frequency 0
    bb = bytearray(b); struct.pack_into("<H", bb, o1, struct.unpack_from("<H", b, o1)[0] + 1); bad.append(bb)  # sum
    bb = bytearray(b); struct.pack_into("<I", bb, o1 + 8 + 4, 2); bad.append(bb)              # stream of 2 bytes
    bb = bytearray(b); bb[off + 6] = 11; bad.append(bb)                                       # scale bits
    for k in (4, 13, 8):                                                                      # stream length byte
        bb = bytearray(b); bb[off + 48] = k; bad.append(bb)
    for bb in bad:
        with pytest.raises(zf.ZfError) as e:
            zf.zf_compressed_from_bytes(bytes(bb))
        assert e.value.status == zf.ZF_ECORRUPT
