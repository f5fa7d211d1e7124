"""Float2Int + bit-packing on the GPU (Section 2.1 "Float2Int"; Table 2 pairs
it with bit-packing): float64 columns decode bit for bit -- the same 64-bit
patterns as the column and as the oracle's decode -- through the transfer
pipeline, from HBM-resident bytes and in the batched kernel."""
import numpy as np
import pytest

import oracle
import zf_workloads as W
from gpu_helpers import Gpu, compress, out_specs

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


def _bits(a):
    return np.asarray(a, np.float64).view(np.uint64)


def _cases():
    rng = np.random.default_rng(41)
    prices = W.decimal_prices(3, 5, 0, 300_001)
    mixed = prices[:70_000].copy()
    mixed[::997] = np.nan
    mixed[5::1999] = np.inf
    mixed[6::2003] = -np.inf
    mixed[7::2999] = -0.0
    mixed[11::3001] = 1.0 / 3.0
    mixed[13::5003] = 2.0 ** 60
    yield "prices_2dp", prices, 65536
    yield "prices_4dp", W.decimal_prices(4, 5, 0, 100_000, 4), 16384
    yield "integers", rng.integers(-10**12, 10**12, 50_000).astype(np.float64), 8192
    yield "mixed_exceptions", mixed, 16384
    yield "random_doubles", rng.standard_normal(20_000), 4096      # every row an exception
    yield "one_row", np.array([12.5]), 1024


CASES = list(_cases())


@pytest.fixture(scope="module")
def gpu():
    g = Gpu()
    yield g
    g.close()


@pytest.mark.parametrize("scheme", [zf.ZF_FLOAT2INT, zf.ZF_RAW])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_float_decode_equals_oracle(gpu, scheme, case):
    name, x, cr = case
    h = compress(x, scheme, cr)
    try:
        for resident in (False, True):
            got, = gpu.decode([h], out_specs(x), resident=resident)
            ref = oracle.decode(zf.zf_compressed_bytes(h))
            assert np.array_equal(_bits(ref), _bits(x))
            assert np.array_equal(_bits(got), _bits(ref)), (name, resident)
    finally:
        zf.zf_compressed_free(h)


def test_oracle_encoded_float2int_on_gpu(gpu):
    for name, x, cr in CASES:
        h = zf.zf_compressed_from_bytes(oracle.encode(x, oracle.FLOAT2INT, cr))
        got, = gpu.decode([h], out_specs(x))
        zf.zf_compressed_free(h)
        assert np.array_equal(_bits(got), _bits(x)), name


def test_float2int_in_batched_and_mixed_calls():
    cols = [(CASES[0][1], zf.ZF_FLOAT2INT), (W.sorted_keys(5, 200_000), zf.ZF_DELTA_BP),
            (CASES[3][1], zf.ZF_FLOAT2INT), (W.dates_rle(5, 100_000), zf.ZF_RLE)]
    handles = [compress(x, s, 32768) for x, s in cols]
    specs = [sp for x, s in cols for sp in out_specs(x)]
    try:
        for flags in (0, zf.ZF_KCFG_BATCHED, zf.ZF_KCFG_BATCHED | zf.ZF_KCFG_GRAPH):
            g = Gpu(stage_bytes=1 << 20, flags=flags)
            try:
                for rep in range(2):
                    got = g.decode(handles, specs)
                    for (x, s), y in zip(cols, got):
                        assert np.array_equal(y.view(np.uint8), x.view(np.uint8)), (flags, s, rep)
            finally:
                g.close()
    finally:
        for h in handles:
            zf.zf_compressed_free(h)


def test_float2int_full_size_column(gpu):
    """64M prices in 1M-row chunks: the whole column bit for bit, and sampled
    chunks against the oracle's own decode of the library's bytes."""
    x = W.decimal_prices(1, 7, 0, 1 << 26)
    h = compress(x, zf.ZF_FLOAT2INT, 1 << 20)
    try:
        got, = gpu.decode([h], out_specs(x))
        assert np.array_equal(_bits(got), _bits(x))
        b = zf.zf_compressed_bytes(h)
        orc = oracle.default()
        for c in (0, 17, 63):
            off, ln, r0, rows = orc.chunk_span(b, c)
            ref = orc.decode_chunk(b[off:off + ln], np.float64)
            assert np.array_equal(_bits(ref), _bits(got[r0:r0 + rows]))
    finally:
        zf.zf_compressed_free(h)


def _f2i_column(e: int, d: np.ndarray) -> bytes:
    """A one-chunk Float2Int column of the integers d at exponent e (no
    exceptions), written from the container layout: FOR reference = min(d),
    packed d - min at b = bits(max - min)."""
    import struct
    ref = int(d.min())
    u = [int(v) - ref for v in d]
    b = max(u).bit_length()
    acc = 0
    for i, v in enumerate(u):
        acc |= v << (i * b)
    packed = acc.to_bytes((len(u) * b + 7) // 8, "little")
    rows = len(d)
    s0 = 64
    s1 = (s0 + len(packed) + 15) // 16 * 16
    blob = bytearray(s1)
    struct.pack_into("<IBBBBIIq", blob, 0, 0x4B48435A, zf.ZF_FLOAT2INT, zf.ZF_F64, b, 0, rows, 0, ref)
    struct.pack_into("<3I3I", blob, 24, s0, s1, s1, len(packed), 0, 0)
    blob[48] = e
    blob[s0:s0 + len(packed)] = packed
    col = bytearray(64 + 32)
    cr = (rows + 1023) // 1024 * 1024
    struct.pack_into("<IHBBIIQQQI", col, 0, 0x4C4F435A, 1, zf.ZF_FLOAT2INT, zf.ZF_F64, 1, cr, rows, 8 * rows,
                     96 + len(blob), 0)
    struct.pack_into("<QQQII", col, 64, 96, len(blob), 0, rows, 0)
    return bytes(col + blob)


def _hard_integers(e: int, rng) -> np.ndarray:
    """Random magnitudes up to 2^53, exact multiples of 5^e, the bounds, and
    the integers nearest to d / 5^e being halfway between two doubles."""
    n = 4000
    bits = rng.integers(1, 54, n)
    a = [int(v) for v in (rng.integers(0, 2**62, n, dtype=np.int64) >> (62 - bits)) + 1]
    p = 5 ** e
    a += [int(k) * p for k in rng.integers(1, max(2, 2**53 // p), 500)]
    a += [1, 2**53, 2**53 - 1, 2**52 + 1] + [10**k for k in range(16)]
    if e:
        for _ in range(1500):
            E = int(rng.integers(-20, 53))
            if 2**E * p > 2**53:
                continue
            num = (2 * int(rng.integers(2**52, 2**53)) + 1) * p
            sh = 53 - E
            base = num >> sh if sh > 0 else num << -sh
            a += [v for v in (base - 1, base, base + 1) if 0 < v <= 2**53]
    a = np.array([min(v, 2**53) for v in a], np.int64)
    sign = rng.integers(0, 2, len(a)) * 2 - 1
    return a * sign


@pytest.mark.parametrize("e", range(19))
def test_float2int_every_exponent_against_the_oracle(gpu, e):
    """The integer-multiply decode equals the oracle's IEEE division d / 10^e
    at every exponent, on the integers where rounding is hardest."""
    d = _hard_integers(e, np.random.default_rng(900 + e))
    buf = _f2i_column(e, d)
    ref = oracle.decode(buf)
    assert np.array_equal(_bits(ref), _bits(d.astype(np.float64) / 10.0 ** e))
    h = zf.zf_compressed_from_bytes(buf)
    try:
        for resident in (False, True):
            got, = gpu.decode([h], [(np.float64, len(d))], resident=resident)
            assert np.array_equal(_bits(got), _bits(ref)), (e, resident)
    finally:
        zf.zf_compressed_free(h)


def test_float2int_integer_beyond_2_53_is_corrupt(gpu):
    for d in (np.array([2**53 + 1, 5], np.int64), np.array([-(2**53) - 1, 0], np.int64)):
        buf = _f2i_column(2, d)
        with pytest.raises(oracle.OracleError):
            oracle.decode(buf)
        h = zf.zf_compressed_from_bytes(buf)
        try:
            gpu.decode([h], [(np.float64, len(d))], expect=zf.ZF_ECORRUPT)
            ok = np.array([2**53, -(2**53)], np.int64)   # the bounds themselves decode
            h2 = zf.zf_compressed_from_bytes(_f2i_column(2, ok))
            got, = gpu.decode([h2], [(np.float64, 2)])
            zf.zf_compressed_free(h2)
            assert np.array_equal(_bits(got), _bits(ok.astype(np.float64) / 100.0))
        finally:
            zf.zf_compressed_free(h)


def _hard_u32(e: int, rng) -> np.ndarray:
    """Integers in [0, 2^32) (so the chunk takes the decoder's 32-bit path):
    random magnitudes, 0, the top of the range, and the integers whose
    quotient by 5^e lies next to a halfway point between two doubles."""
    a = [int(v) for v in rng.integers(0, 2**32, 3000, dtype=np.int64) >> rng.integers(0, 32, 3000)]
    a += [0, 1, 2**32 - 1, 2**31, 5**min(e, 13)]
    p = 5 ** e
    for _ in range(3000):
        E = int(rng.integers(-45, 32))
        if 2**E * p > 2**32:
            continue
        num = (2 * int(rng.integers(2**52, 2**53)) + 1) * p
        sh = 53 - E
        base = num >> sh if sh > 0 else num << -sh
        a += [v for v in (base - 1, base, base + 1) if 0 <= v < 2**32]
    return np.array(a[:4093], np.int64)    # not a multiple of four: a ragged last step


@pytest.mark.parametrize("e", range(1, 19))
def test_float2int_32_bit_path_every_exponent(gpu, e):
    """Chunks whose integers all lie in [0, 2^32) decode through the 32-bit
    integer path; the result equals the oracle's division at every exponent."""
    d = _hard_u32(e, np.random.default_rng(1900 + e))
    assert d.min() == 0 and d.max() == 2**32 - 1
    buf = _f2i_column(e, d)
    ref = oracle.decode(buf)
    assert np.array_equal(_bits(ref), _bits(d.astype(np.float64) / 10.0 ** e))
    h = zf.zf_compressed_from_bytes(buf)
    try:
        for resident in (False, True):
            got, = gpu.decode([h], [(np.float64, len(d))], resident=resident)
            assert np.array_equal(_bits(got), _bits(ref)), (e, resident)
    finally:
        zf.zf_compressed_free(h)
