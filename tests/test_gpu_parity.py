"""GPU decode parity: every decode through the C ABI equals the original
column and the oracle's decode, element by element (bit-exact integers)."""
import numpy as np
import pytest

import oracle
import zf_workloads as W
from gpu_helpers import Gpu, compress, out_specs

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    g = Gpu()
    yield g
    g.close()


def _cases():
    I32, I64 = np.int32, np.int64
    rng = np.random.default_rng(21)
    yield "uniform12", W.uniform_int(1, 0, 0, 300001, 0, 4096).astype(I32), 65536
    yield "keys", W.sorted_keys(3, 400000), 131072
    yield "dates", W.dates_rle(3, 400000), 131072
    yield "dict25", W.dict_codes(3, 7, 0, 150000), 32768
    yield "lognormal", W.lognormal_cents(3, 9, 0, 150000), 32768
    yield "i32_extremes", np.array([2**31 - 1, -2**31, 0, -1, 5] * 999, I32), 1024
    yield "i64_extremes", np.array([2**63 - 1, -2**63, 0, -1, 5] * 999, I64), 2048
    yield "wide64", (rng.integers(-2**62, 2**62, 20000, dtype=I64) * 2 + 1), 8192
    yield "ragged", rng.integers(-1000, 1000, 12345).astype(I64), 4096
    yield "constant", np.full(5000, 42, I32), 1024
    yield "one_row", np.array([7], I64), 1024
    yield "outlier_runs", W.rle_distribution(2, "outlier", 70000, 64, 1024), 16384
    yield "mixed_runs", W.rle_distribution(2, "mixed", 70000, 4, 32), 16384
    yield "random_runs", W.rle_distribution(2, "random", 70000, 1, 64), 16384
    yield "one_long_run", np.full(300000, -9, I32), 131072


CASES = list(_cases())


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_for_every_bit_width(gpu, dtype):
    """FOR + bit-packing at every width b (0..32 for int32, 0..64 for int64),
    each chunk spanning its full range so that b = bits(max - min); ragged
    chunk and tile ends; every width path of the decoder (two-word, three-word
    window, one extraction per value) against the column and the oracle."""
    rng = np.random.default_rng(61)
    top = 32 if dtype == np.int32 else 64
    parts = []
    for b in range(0, top + 1):
        n = 3000 + 37 * b
        lo = -(1 << (top - 1))
        span = (1 << b) - 1
        v = rng.integers(0, 1 << min(b, 62), n, dtype=np.uint64) if b else np.zeros(n, np.uint64)
        if b > 62:
            v = v * (1 << (b - 62)) + rng.integers(0, 1 << (b - 62), n, dtype=np.uint64)
        v[0], v[-1] = 0, span
        parts.append((np.uint64(lo & ((1 << 64) - 1)) + v).view(np.int64).astype(dtype) if top == 64 else
                     (v.astype(np.int64) + lo).astype(dtype))
    for b, x in enumerate(parts):
        h = compress(x, zf.ZF_FOR_BP, 1024 * (1 + b % 3))
        try:
            from oracle_pins import chunks_of
            assert chunks_of(oracle.default(), zf.zf_compressed_bytes(h))[0][4]["bw"] == b
            for resident in (False, True):
                got, = gpu.decode([h], out_specs(x), resident=resident)
                assert np.array_equal(got, x), (b, resident)
        finally:
            zf.zf_compressed_free(h)


@pytest.mark.parametrize("dtype", [np.int32, np.int64])
def test_dict_every_code_width(gpu, dtype):
    """Dictionary + bit-packing with 2^(b-1) + 1 distinct values, so the
    codes are b = 1..16 bits wide, on ragged chunks, against the column."""
    rng = np.random.default_rng(62)
    for b in range(1, 17):
        nd = (1 << (b - 1)) + 1
        vals = rng.integers(-(1 << 31), 1 << 31, nd).astype(dtype) * (3 if dtype == np.int64 else 1)
        vals = np.unique(vals)
        x = vals[np.concatenate([np.arange(len(vals)), rng.integers(0, len(vals), 5000 + 41 * b)])]
        h = compress(x, zf.ZF_DICT_BP, 1 << 20)
        try:
            got, = gpu.decode([h], out_specs(x))
            assert np.array_equal(got, x), b
        finally:
            zf.zf_compressed_free(h)


@pytest.mark.parametrize("scheme", ["raw", "for_bp", "dict_bp", "delta_bp", "rle"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_decode_equals_oracle(gpu, scheme, case):
    name, x, cr = case
    s = oracle.SCHEMES[scheme]
    try:
        h = compress(x, s, cr)
    except zf.ZfError:
        assert scheme == "dict_bp"
        return
    try:
        got, = gpu.decode([h], out_specs(x))
        ref = oracle.decode(zf.zf_compressed_bytes(h))
        assert np.array_equal(ref, x)
        assert np.array_equal(got, ref)
    finally:
        zf.zf_compressed_free(h)


def test_oracle_encoded_streams_decode_on_gpu(gpu):
    for name, x, cr in CASES[:6]:
        for s in (oracle.FOR_BP, oracle.DELTA_BP, oracle.RLE):
            h = zf.zf_compressed_from_bytes(oracle.encode(x, s, cr))
            got, = gpu.decode([h], out_specs(x))
            zf.zf_compressed_free(h)
            assert np.array_equal(got, x), (name, s)


def test_lz77_strings(gpu):
    t, o = W.text_column(7, 1000003)
    for enc in ("library", "oracle"):
        if enc == "library":
            h = compress(t, zf.ZF_LZ77, offsets=o)
        else:
            h = zf.zf_compressed_from_bytes(oracle.encode_strings(t, o))
        got_t, got_o = gpu.decode([h], out_specs(t, o))
        zf.zf_compressed_free(h)
        assert np.array_equal(got_t, t), enc
        assert np.array_equal(got_o, o), enc


def test_raw_string_columns(gpu):
    """A string column stored raw (the selector's other class for bytes):
    every byte of each 64 KiB chunk comes back, through the transfer, the
    resident and the batched paths."""
    t, o = W.text_column(8, 300001)                  # ragged last chunk
    h = compress(t, zf.ZF_RAW, offsets=o)
    try:
        for resident in (False, True):
            got_t, got_o = gpu.decode([h], out_specs(t, o), resident=resident)
            assert np.array_equal(got_t, t), resident
            assert np.array_equal(got_o, o), resident
    finally:
        zf.zf_compressed_free(h)
    g = Gpu(flags=zf.ZF_KCFG_BATCHED)
    h = compress(t, zf.ZF_RAW, offsets=o)
    try:
        got_t, got_o = g.decode([h], out_specs(t, o))
        assert np.array_equal(got_t, t) and np.array_equal(got_o, o)
    finally:
        zf.zf_compressed_free(h)
        g.close()


def test_strdict_strings(gpu):
    """String dictionary + bit-packing: library- and oracle-encoded text
    columns, ragged chunks, long and byte-heavy tokens, through the transfer,
    resident and batched paths."""
    rng = np.random.default_rng(12)
    raw = rng.integers(0, 256, 150000).astype(np.uint8)
    # 64-byte tokens (63 letters and a space) between short ones: batches of 64
    # tokens that go through the output window in four rounds
    lw = rng.integers(97, 123, (3000, 64)).astype(np.uint8)
    lw[:, 63] = 32
    lw[::7, 3] = 32                                   # every seventh word cut short
    longs = lw.reshape(-1)
    # words of 12-40 bytes: 64-token batches of 1-2.5 KB (two rounds through the window)
    wl = rng.integers(12, 41, 6000)
    mids = rng.integers(97, 123, int(wl.sum())).astype(np.uint8)
    mids[np.cumsum(wl) - 1] = 32
    cases = [(W.text_column(7, 1000003), 1 << 20), (W.text_column(8, 300001), 65536),
             ((raw, np.array([0, 70000, 70000, 150000], np.int32)), 131072),
             ((longs, np.array([0, 5, 64 * 1000 + 1, longs.size], np.int32)), 65536),
             ((mids, np.array([0, mids.size], np.int32)), 65536),
             ((np.frombuffer(b"xyz", np.uint8).copy(), np.array([0, 3], np.int32)), 65536)]
    for (t, o), cb in cases:
        for enc in ("library", "oracle"):
            if enc == "library":
                col = zf.Column(t, o)
                h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_STRDICT, chunk_rows=cb), col)
            else:
                h = zf.zf_compressed_from_bytes(oracle.encode_strings(t, o, cb, scheme=oracle.STRDICT))
            try:
                for resident in (False, True):
                    got_t, got_o = gpu.decode([h], out_specs(t, o), resident=resident)
                    assert np.array_equal(got_t, t), (enc, cb, resident)
                    assert np.array_equal(got_o, o), (enc, cb, resident)
            finally:
                zf.zf_compressed_free(h)
    t, o = cases[0][0]
    g = Gpu(flags=zf.ZF_KCFG_BATCHED)
    h = zf.zf_compressed_from_bytes(oracle.encode_strings(t, o, 1 << 18, scheme=oracle.STRDICT))
    try:
        got_t, got_o = g.decode([h], out_specs(t, o))
        assert np.array_equal(got_t, t) and np.array_equal(got_o, o)
    finally:
        zf.zf_compressed_free(h)
        g.close()


def test_strdict_dictionary_larger_than_l1(gpu):
    """A chunk of 30,000 distinct 12-byte words (a dictionary of about
    500 KB, far more than an SM's L1) in a column with small-dictionary
    chunks decodes exactly on the transfer, resident and batched paths."""
    rng = np.random.default_rng(44)
    letters = rng.integers(97, 123, (30000, 11)).astype(np.uint8)
    words = np.concatenate([letters, np.full((30000, 1), 32, np.uint8)], 1)   # 12-byte tokens "xxxxxxxxxxx "
    big = words[rng.permutation(30000)].reshape(-1)[: 1 << 20]                 # 1 MiB: every word about once
    small, so = W.text_column(10, 1 << 20)
    t = np.concatenate([big, small])
    o = np.concatenate([np.arange(0, big.size, 120, dtype=np.int64), big.size + so.astype(np.int64)]).astype(np.int32)
    o = np.unique(o)
    col = zf.Column(t, o)
    h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_STRDICT, chunk_rows=1 << 20), col)
    try:
        from oracle_pins import chunks_of
        chs = chunks_of(oracle.default(), zf.zf_compressed_bytes(h))
        assert chs[0][4]["n_aux"] > 20000 and chs[-1][4]["n_aux"] < 20000
        for resident in (False, True):
            got_t, got_o = gpu.decode([h], out_specs(t, o), resident=resident)
            assert np.array_equal(got_t, t) and np.array_equal(got_o, o), resident
        g = Gpu(flags=zf.ZF_KCFG_BATCHED)
        try:
            got_t, got_o = g.decode([h], out_specs(t, o))
            assert np.array_equal(got_t, t) and np.array_equal(got_o, o)
        finally:
            g.close()
    finally:
        zf.zf_compressed_free(h)


def test_strdict_device_detects_corrupt_streams(gpu):
    """A code past the dictionary, and a tile start that the lengths do not
    reach (both pass the host's structural checks): ZF_ECORRUPT, no fault."""
    import struct
    from oracle_pins import chunks_of
    t, o = W.text_column(9, 400000)
    b = oracle.encode_strings(t, o, 1 << 18, scheme=oracle.STRDICT)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    nd, bw = ch["n_aux"], ch["bw"]
    assert nd < (1 << bw)                                   # a free code exists above the dictionary
    c2 = off + ch["offs"][2]
    def code_past_dictionary(bb):
        w = int.from_bytes(bb[c2:c2 + 4], "little")
        w = (w & ~((1 << bw) - 1)) | ((1 << bw) - 1)        # token 0 takes the largest code
        bb[c2:c2 + 4] = w.to_bytes(4, "little")
    tile1 = off + ch["offs"][0] + 4 * (nd + 2)              # start of the second 1024-token tile
    def tile_start_plus_one(bb):
        struct.pack_into("<I", bb, tile1, struct.unpack_from("<I", bb, tile1)[0] + 1)
    for fn in (code_past_dictionary, tile_start_plus_one):
        h = zf.zf_compressed_from_bytes(_corrupt(b, fn))
        try:
            gpu.decode([h], out_specs(t, o), expect=zf.ZF_ECORRUPT)
        finally:
            zf.zf_compressed_free(h)
    h = zf.zf_compressed_from_bytes(b)                      # the context stays usable
    try:
        got_t, got_o = gpu.decode([h], out_specs(t, o))
        assert np.array_equal(got_t, t) and np.array_equal(got_o, o)
    finally:
        zf.zf_compressed_free(h)


@pytest.mark.parametrize("stream_rows", [32, 64, 128, 256, 512, 1024, 2048, 4096])
def test_ans_stream_lengths(gpu, stream_rows):
    """Every stream length of the format (2^5..2^12 rows per rANS stream,
    header byte 48): library bytes equal the oracle's, and the GPU decode of
    both equals the column, on ragged chunks whose last stream is short, an
    int64 column of 256 values, and a chunk with fewer rows than a stream."""
    rng = np.random.default_rng(700 + stream_rows)
    cases = [
        (rng.choice([65, 78, 82], 130003, p=[0.25, 0.5, 0.25]).astype(np.int32), 1 << 16),
        (rng.integers(-(1 << 63), (1 << 63) - 1, 256, dtype=np.int64)[rng.integers(0, 256, 40001)], 8192),
        (rng.integers(0, 3, 17).astype(np.int32), 1024),
    ]
    for x, cr in cases:
        col = zf.Column(x)
        h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS, chunk_rows=cr,
                                           ans_stream_rows=stream_rows), col)
        try:
            ob = oracle.encode(x, oracle.ANS, cr, ans_stream_rows=stream_rows)
            assert zf.zf_compressed_bytes(h) == ob
            for resident in (False, True):
                got, = gpu.decode([h], out_specs(x), resident=resident)
                assert np.array_equal(got, x), (stream_rows, cr, resident)
        finally:
            zf.zf_compressed_free(h)


def test_ans_columns(gpu):
    """Dictionary + ANS: library- and oracle-encoded low-cardinality columns
    (ragged chunks and streams, one value, 256 values, type extremes) through
    the transfer, resident and batched paths; a flipped stream byte is
    reported, and the context stays usable."""
    rng = np.random.default_rng(31)
    cases = [
        (rng.choice([65, 78, 82], 300001, p=[0.25, 0.5, 0.25]).astype(np.int32), 1 << 17),
        (rng.integers(-(1 << 63), (1 << 63) - 1, 256, dtype=np.int64)[rng.integers(0, 256, 70000)], 16384),
        (np.full(5000, 7, np.int64), 4096),
        (np.array([-2**31, 2**31 - 1] * 3001, np.int32), 2048),
        ((rng.geometric(0.05, 200003) % 256).astype(np.int32), 1 << 20),
        # four values (the largest alphabet decoded from cumulative frequencies
        # in registers, one of them rare) and five (the first with the slot table)
        (np.array([-2**63, 2**63 - 1, 0, 77], np.int64)[rng.choice(4, 90001, p=[0.6, 0.3, 0.0995, 0.0005])], 32768),
        (np.array([3, 1, 4, 1 << 30, -5], np.int32)[rng.integers(0, 5, 70001)], 16384),
    ]
    for x, cr in cases:
        for enc in ("library", "oracle"):
            if enc == "library":
                col = zf.Column(x)
                h = zf.zf_compress_host(zf.zf_plan(None, col, scheme=zf.ZF_ANS, chunk_rows=cr), col)
            else:
                h = zf.zf_compressed_from_bytes(oracle.encode(x, oracle.ANS, cr))
            try:
                for resident in (False, True):
                    got, = gpu.decode([h], out_specs(x), resident=resident)
                    assert np.array_equal(got, x), (enc, cr, resident)
            finally:
                zf.zf_compressed_free(h)
    x, cr = cases[0]
    g = Gpu(flags=zf.ZF_KCFG_BATCHED)
    h = zf.zf_compressed_from_bytes(oracle.encode(x, oracle.ANS, cr))
    h2 = compress(W.sorted_keys(3, 100000), zf.ZF_DELTA_BP, 65536)       # a mixed call
    try:
        got, got2 = g.decode([h, h2], out_specs(x) + out_specs(W.sorted_keys(3, 100000)))
        assert np.array_equal(got, x) and np.array_equal(got2, W.sorted_keys(3, 100000))
    finally:
        zf.zf_compressed_free(h)
        zf.zf_compressed_free(h2)
        g.close()
    from oracle_pins import chunks_of
    b = oracle.encode(x, oracle.ANS, cr)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    bad = _corrupt(b, lambda bb: bb.__setitem__(off + ch["offs"][2] + 9, bb[off + ch["offs"][2] + 9] ^ 0x21))
    h = zf.zf_compressed_from_bytes(bad)
    try:
        gpu.decode([h], out_specs(x), expect=zf.ZF_ECORRUPT)
    finally:
        zf.zf_compressed_free(h)
    h = zf.zf_compressed_from_bytes(b)
    try:
        got, = gpu.decode([h], out_specs(x))
        assert np.array_equal(got, x)
    finally:
        zf.zf_compressed_free(h)


def test_lz77_edge_blocks(gpu):
    cases = [
        np.frombuffer(b"a" * 70000, np.uint8),                            # one long overlapping run
        np.frombuffer((b"abc" * 40000)[:100000], np.uint8),               # offset 3 overlap
        W.uniform_int(9, 1, 0, 150000, 0, 256).astype(np.uint8),          # incompressible: raw blocks
        np.frombuffer(b"xyz", np.uint8),                                   # tiny
    ]
    for t in cases:
        t = np.ascontiguousarray(t)
        o = np.array([0, len(t)], np.int32)
        h = compress(t, zf.ZF_LZ77, offsets=o)
        got_t, got_o = gpu.decode([h], out_specs(t, o))
        zf.zf_compressed_free(h)
        assert np.array_equal(got_t, t)
        assert np.array_equal(got_o, o)


def test_empty_column(gpu):
    x = np.zeros(0, np.int32)
    h = compress(x, zf.ZF_FOR_BP, 1024)
    got, = gpu.decode([h], [(np.int32, 0)])
    zf.zf_compressed_free(h)
    assert len(got) == 0


@pytest.mark.parametrize("tile_rows,threads", [(1024, 128), (2048, 256), (4096, 512), (8192, 256), (16384, 512)])
def test_schedule_invariance(tile_rows, threads):
    """Every kernel geometry decodes the same bytes (Section 4: a <L,S,C>
    tuple changes the schedule, not the computation)."""
    g = Gpu(tile_rows=tile_rows, threads=threads, stage_bytes=1 << 20)
    try:
        for name, x, cr in (CASES[0], CASES[1], CASES[2], CASES[11], CASES[4]):
            for s in (zf.ZF_FOR_BP, zf.ZF_DELTA_BP, zf.ZF_RLE):
                h = compress(x, s, cr)
                got, = g.decode([h], out_specs(x))
                zf.zf_compressed_free(h)
                assert np.array_equal(got, x), (name, s, tile_rows, threads)
    finally:
        g.close()


def test_batched_mixed_columns_and_resident():
    cols = [(CASES[0][1], zf.ZF_FOR_BP), (CASES[1][1], zf.ZF_DELTA_BP), (CASES[2][1], zf.ZF_RLE),
            (CASES[3][1], zf.ZF_DICT_BP), (CASES[4][1], zf.ZF_FOR_BP), (CASES[5][1], zf.ZF_RAW)]
    handles = [compress(x, s, 65536) for x, s in cols]
    specs = [sp for x, s in cols for sp in out_specs(x)]
    try:
        for flags, resident in ((0, False), (zf.ZF_KCFG_BATCHED, False), (zf.ZF_KCFG_BATCHED, True), (0, True)):
            g = Gpu(stage_bytes=1 << 19, flags=flags)
            try:
                got = g.decode(handles, specs, resident=resident)
                for (x, s), y in zip(cols, got):
                    assert np.array_equal(y, x), (flags, resident, s)
            finally:
                g.close()
    finally:
        for h in handles:
            zf.zf_compressed_free(h)


def test_ring_slots_and_small_stages():
    x = W.sorted_keys(5, 1 << 20)
    h = compress(x, zf.ZF_DELTA_BP, 65536)
    try:
        for slots in (2, 3, 8):
            g = Gpu(stage_bytes=40000)
            zf.zf_ctx_set_ring(g.ctx, slots)
            got, = g.decode([h], out_specs(x))
            assert g.last_stats.n_stages > slots
            g.close()
            assert np.array_equal(got, x)
    finally:
        zf.zf_compressed_free(h)


def test_api_misuse(gpu):
    torch = gpu.torch
    x = W.sorted_keys(5, 10000)
    h = compress(x, zf.ZF_DELTA_BP, 4096)
    buf = torch.empty(x.nbytes + 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(zf.ZfError) as e:  # too small
        zf.zf_transfer_decompress(gpu.ctx, [h], [buf.data_ptr()], [x.nbytes - 8])
    assert e.value.status == zf.ZF_EINVAL
    with pytest.raises(zf.ZfError) as e:  # misaligned
        zf.zf_transfer_decompress(gpu.ctx, [h], [buf.data_ptr() + 4], [x.nbytes])
    assert e.value.status == zf.ZF_EINVAL
    zf.zf_transfer_decompress(gpu.ctx, [h], [buf.data_ptr()], [buf.numel()])
    with pytest.raises(zf.ZfError) as e:  # not synced
        zf.zf_transfer_decompress(gpu.ctx, [h], [buf.data_ptr()], [buf.numel()])
    assert e.value.status == zf.ZF_EBUSY
    zf.zf_sync(gpu.ctx)
    zf.zf_compressed_free(h)
    assert np.array_equal(buf[: x.nbytes].cpu().numpy().view(np.int64), x)


def _corrupt(b: bytes, fn) -> bytes:
    bb = bytearray(b)
    fn(bb)
    return bytes(bb)


def test_device_detects_rle_lengths_that_wrap_32_bits(gpu):
    """A 64M-row RLE chunk whose first tile's 1,024 run lengths each pass the
    per-run check (1 <= length <= rows) but add up to 2^32 + 1,024: a 32-bit
    sum would wrap to the tile's 1,024 rows.  The device reports ZF_ECORRUPT."""
    import struct
    from oracle_pins import chunks_of
    n = 1 << 26
    x = np.full(n, 5000, np.int32)
    x[:1024] = np.arange(1024)                       # runs 0..1023 of length 1, then one long run
    b = oracle.encode(x, oracle.RLE, n)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    lo = off + ch["offs"][1]                          # run lengths
    lens = [(1 << 25) + 1, (1 << 25) - 1] + [1 << 25] * 126 + [1] * 895 + [129]
    assert len(lens) == 1024 and sum(lens) == (1 << 32) + 1024
    bad = _corrupt(b, lambda bb: struct.pack_into("<1024I", bb, lo, *lens))
    h = zf.zf_compressed_from_bytes(bad)
    try:
        gpu.decode([h], out_specs(x), expect=zf.ZF_ECORRUPT)
    finally:
        zf.zf_compressed_free(h)


def test_device_detects_corrupt_streams(gpu):
    """Streams that pass the host's structural checks but whose data is
    inconsistent make the decoder report ZF_ECORRUPT, without a fault."""
    import struct
    from oracle_pins import chunks_of
    x = W.dates_rle(9, 50000)
    b = oracle.encode(x, oracle.RLE, 16384)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[1]
    lo = off + ch["offs"][1]
    bad = _corrupt(b, lambda bb: struct.pack_into("<I", bb, lo + 8, struct.unpack_from("<I", bb, lo + 8)[0] + 1))
    h = zf.zf_compressed_from_bytes(bad)
    gpu.decode([h], out_specs(x), expect=zf.ZF_ECORRUPT)
    zf.zf_compressed_free(h)
    # a zero run length
    bad = _corrupt(b, lambda bb: struct.pack_into("<I", bb, lo + 4, 0))
    h = zf.zf_compressed_from_bytes(bad)
    gpu.decode([h], out_specs(x), expect=zf.ZF_ECORRUPT)
    zf.zf_compressed_free(h)
    # a dictionary code past the dictionary (3 values -> b = 2 -> code 3 is free)
    d = np.array([10, 20, 30, 10] * 1000, np.int32)
    b = oracle.encode(d, oracle.DICT_BP, 4096)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    bad = _corrupt(b, lambda bb: bb.__setitem__(off + ch["offs"][1], 0xFF))
    h = zf.zf_compressed_from_bytes(bad)
    gpu.decode([h], out_specs(d), expect=zf.ZF_ECORRUPT)
    zf.zf_compressed_free(h)
    # an LZ77 offset beyond the bytes produced so far
    t = np.frombuffer(b"abcdabcdabcdabcd" * 100, np.uint8).copy()
    o = np.array([0, len(t)], np.int32)
    b = oracle.encode_strings(t, o)
    off, ln, r0, rows, ch = chunks_of(oracle.default(), b)[0]
    bad = _corrupt(b, lambda bb: struct.pack_into("<H", bb, off + ch["offs"][1], 9000))
    h = zf.zf_compressed_from_bytes(bad)
    gpu.decode([h], out_specs(t, o), expect=zf.ZF_ECORRUPT)
    zf.zf_compressed_free(h)
    # an LZ77 length of four LEB128 bytes (at most three are allowed)
    def four_byte_length(bb):
        p = off + ch["offs"][0]
        bb[p:p + 4] = bytes([0x80, 0x80, 0x80, 0x00])
    h = zf.zf_compressed_from_bytes(_corrupt(b, four_byte_length))
    gpu.decode([h], out_specs(t, o), expect=zf.ZF_ECORRUPT)
    zf.zf_compressed_free(h)
    # the context stays usable after a reported error
    h = compress(x, zf.ZF_RLE, 16384)
    got, = gpu.decode([h], out_specs(x))
    zf.zf_compressed_free(h)
    assert np.array_equal(got, x)
