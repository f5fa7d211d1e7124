"""Parity at the full sizes of the benchmark workloads, in the launch
configuration the benchmark uses: the whole decode is compared with the
generated column, and sampled chunks with the oracle's own decode."""
import numpy as np
import pytest

import oracle
import zf_workloads as W
from gpu_helpers import Gpu, compress, out_specs

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


def _sampled_oracle_check(h, got, dtype, samples=(0, 1, -1)):
    b = zf.zf_compressed_bytes(h)
    info = oracle.column_info(b)
    for s in samples:
        c = s % info["n_chunks"]
        off, ln, r0, rows = oracle.chunk_span(b, c)
        ref = oracle.decode_chunk(b[off:off + ln], dtype)
        assert np.array_equal(got[r0:r0 + rows], ref), c


def test_fully_parallel_1m_int32_for12():
    """1,048,576 int32 uniform on [0,4096), FOR + 12-bit packing, 65,536-row chunks, seeds 1-3."""
    g = Gpu()
    try:
        for seed in (1, 2, 3):
            x = W.uniform_int(seed, 0, 0, 1 << 20, 0, 4096).astype(np.int32)
            h = compress(x, zf.ZF_FOR_BP, 65536)
            raw, comp, nch = zf.zf_compressed_info(h)
            assert nch == 16 and comp == 64 + 32 * 16 + 16 * (64 + 98304)
            got, = g.decode([h], out_specs(x))
            assert np.array_equal(got, x)
            _sampled_oracle_check(h, got, np.int32, samples=range(16))
            zf.zf_compressed_free(h)
    finally:
        g.close()


def test_group_parallel_64m_keys_and_dates():
    """64M sorted int64 keys (delta) and 64M int32 dates (RLE), 1M-row chunks, one call."""
    n = 1 << 26
    keys = W.sorted_keys(1, n)
    dates = W.dates_rle(1, n)
    hk = compress(keys, zf.ZF_DELTA_BP, 1 << 20)
    hd = compress(dates, zf.ZF_RLE, 1 << 20)
    g = Gpu()
    try:
        for resident in (False, True):
            gk, gd = g.decode([hk, hd], out_specs(keys) + out_specs(dates), resident=resident)
            assert np.array_equal(gk, keys)
            assert np.array_equal(gd, dates)
        _sampled_oracle_check(hk, gk, np.int64)
        _sampled_oracle_check(hd, gd, np.int32)
    finally:
        g.close()
        zf.zf_compressed_free(hk)
        zf.zf_compressed_free(hd)


def test_non_parallel_256mb_text():
    """268,435,456 bytes of Zipf(1.1) words, LZ77 in 64 KiB blocks, offsets delta-packed."""
    t, o = W.text_column(1, 1 << 28)
    h = compress(t, zf.ZF_LZ77, offsets=o)
    g = Gpu()
    try:
        gt, go = g.decode([h], out_specs(t, o))
        assert np.array_equal(gt, t)
        assert np.array_equal(go, o)
        b = zf.zf_compressed_bytes(h)
        info = oracle.column_info(b)
        for c in (0, 1, 1000, info["n_chunks"] - 1):
            off, ln, r0, rows = oracle.chunk_span(b, c)
            assert np.array_equal(gt[r0:r0 + rows], oracle.decode_chunk(b[off:off + ln], np.uint8))
    finally:
        g.close()
        zf.zf_compressed_free(h)


def test_single_64m_row_chunks():
    """Chunks far above the default size: one 64M-row chunk per column
    (512 MiB of int64 keys, 256 MiB of int32 dates and FOR values), so row
    and byte offsets inside a chunk run into the hundreds of millions."""
    n = 1 << 26
    cols = [(W.sorted_keys(7, n), zf.ZF_DELTA_BP),
            (W.dates_rle(7, n), zf.ZF_RLE),
            (W.uniform_int(7, 0, 0, n, 0, 4096).astype(np.int32), zf.ZF_FOR_BP)]
    g = Gpu()
    try:
        for x, s in cols:
            h = compress(x, s, n)
            try:
                assert zf.zf_compressed_info(h)[2] == 1
                for resident in (False, True):
                    got, = g.decode([h], out_specs(x), resident=resident)
                    assert np.array_equal(got, x), (s, resident)
                _sampled_oracle_check(h, got, x.dtype, samples=(0,))
            finally:
                zf.zf_compressed_free(h)
    finally:
        g.close()
