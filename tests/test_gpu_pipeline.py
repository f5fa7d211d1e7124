"""The pipeline's replay and tuning paths: a transfer captured once as a
CUDA graph and replayed, and the exhaustive geometry search (Section 4,
Table 3's brute-force search) visiting every point once and keeping the
fastest."""
import numpy as np
import pytest

import zf_workloads as W
from gpu_helpers import Gpu, compress, out_specs

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def columns():
    cols = [(W.sorted_keys(21, 3 << 20), zf.ZF_DELTA_BP, 1 << 18),
            (W.dates_rle(21, 3 << 20), zf.ZF_RLE, 1 << 18),
            (W.uniform_int(21, 0, 0, 2_000_000, 0, 4096).astype(np.int32), zf.ZF_FOR_BP, 65536),
            (W.dict_codes(21, 5, 0, 1_000_000), zf.ZF_DICT_BP, 65536)]
    hs = [compress(x, s, cr) for x, s, cr in cols]
    yield cols, hs
    for h in hs:
        zf.zf_compressed_free(h)


@pytest.mark.parametrize("flags", [zf.ZF_KCFG_GRAPH, zf.ZF_KCFG_GRAPH | zf.ZF_KCFG_BATCHED])
def test_graph_replay(columns, flags):
    cols, hs = columns
    specs = [sp for x, s, cr in cols for sp in out_specs(x)]
    g = Gpu(stage_bytes=4 << 20, flags=flags)
    try:
        bufs = g.alloc(specs)
        outs, caps = [b.data_ptr() for b in bufs], [b.numel() for b in bufs]
        for rep in range(3):                      # capture once, then replay
            for b in bufs:
                b.fill_(0x5A)
            g.torch.cuda.synchronize()            # the library runs on its own streams
            zf.zf_transfer_decompress(g.ctx, hs, outs, caps)
            st, stats = zf.zf_sync(g.ctx)
            assert stats.n_stages > 2
            for (x, s, cr), b in zip(cols, bufs):
                assert np.array_equal(b[: x.nbytes].cpu().numpy().view(x.dtype), x), (rep, s)
        bufs2 = g.alloc(specs)                    # new outputs: a new capture
        zf.zf_transfer_decompress(g.ctx, hs, [b.data_ptr() for b in bufs2], [b.numel() for b in bufs2])
        zf.zf_sync(g.ctx)
        for (x, s, cr), b in zip(cols, bufs2):
            assert np.array_equal(b[: x.nbytes].cpu().numpy().view(x.dtype), x)
    finally:
        g.close()


@pytest.mark.parametrize("transfer,npts", [(False, 15), (True, 150)])
def test_tune_visits_every_point_and_keeps_the_fastest(columns, transfer, npts):
    cols, hs = columns
    specs = [sp for x, s, cr in cols for sp in out_specs(x)]
    g = Gpu()
    try:
        bufs = g.alloc(specs)
        outs, caps = [b.data_ptr() for b in bufs], [b.numel() for b in bufs]
        pts, best = zf.zf_tune(g.ctx, hs, outs, caps, transfer=transfer, reps=2)
        assert len(pts) == npts
        seen = {(p.kcfg.tile_rows, p.kcfg.threads, p.kcfg.stage_bytes, p.kcfg.flags & zf.ZF_KCFG_GRAPH) for p in pts}
        assert len(seen) == npts
        fastest = min(pts, key=lambda p: p.ms)
        assert (best.tile_rows, best.threads) == (fastest.kcfg.tile_rows, fastest.kcfg.threads)
        if transfer:
            # stage size and graph replay are searched too, the transfer timed as its caller sees it
            assert best.stage_bytes == fastest.kcfg.stage_bytes
            assert best.flags & zf.ZF_KCFG_GRAPH == fastest.kcfg.flags & zf.ZF_KCFG_GRAPH
            assert {p.kcfg.flags & zf.ZF_KCFG_GRAPH for p in pts} == {0, zf.ZF_KCFG_GRAPH}
        # the context now decodes with the chosen geometry, bit-exact
        for b in bufs:
            b.fill_(0)
        g.torch.cuda.synchronize()
        zf.zf_transfer_decompress(g.ctx, hs, outs, caps)
        zf.zf_sync(g.ctx)
        for (x, s, cr), b in zip(cols, bufs):
            assert np.array_equal(b[: x.nbytes].cpu().numpy().view(x.dtype), x)
    finally:
        g.close()


def test_tune_of_one_class_is_kept_for_that_class(columns):
    """Tuning columns of one (scheme, dtype, bit-width bucket) class records
    the fastest geometry for that class and leaves the context automatic:
    other classes keep the built-in geometry, and decodes stay bit-exact."""
    cols, hs = columns
    g = Gpu()
    try:
        (x, s, cr), h = cols[0], hs[0]                 # the delta keys
        assert s == zf.ZF_DELTA_BP
        before = zf.zf_ctx_tuned_geometry(g.ctx, zf.ZF_DELTA_BP, zf.ZF_I64, 8)
        buf = g.alloc(out_specs(x))[0]
        pts, best = zf.zf_tune(g.ctx, [h], [buf.data_ptr()], [buf.numel()], transfer=False, reps=2)
        assert len(pts) == 15
        # the class of these chunks (bucket of the column's widest delta width) has the tuned geometry
        geo = [zf.zf_ctx_tuned_geometry(g.ctx, zf.ZF_DELTA_BP, zf.ZF_I64, w) for w in (8, 16, 32, 64)]
        assert any((k.tile_rows, k.threads) == (best.tile_rows, best.threads) for k in geo)
        # RLE int32 is another class: still the built-in geometry
        rle = zf.zf_ctx_tuned_geometry(g.ctx, zf.ZF_RLE, zf.ZF_I32, 0)
        assert (rle.tile_rows, rle.threads) == (4096, 128)
        assert (before.tile_rows, before.threads) == (2048, 128)
        # decoding every column afterwards is exact
        for (x2, s2, cr2), h2 in zip(cols, hs):
            got, = g.decode([h2], out_specs(x2))
            assert np.array_equal(got, x2)
    finally:
        g.close()


def test_measured_rates_for_johnsons_rule(columns):
    """zf_measure_copy records the link rate of the call's own pieces and a
    resident zf_tune of one class records that class's decode rate: the rates
    the transfer's Johnson ordering (Section 3.3) reads; a transfer in that
    order, in the order given and in reverse all decode exactly."""
    cols, hs = columns
    g = Gpu()
    try:
        assert zf.zf_ctx_rates(g.ctx, zf.ZF_DELTA_BP, zf.ZF_I64, 8) == (0.0, 0.0)
        ms = zf.zf_measure_copy(g.ctx, hs, 3)
        comp = sum(zf.zf_compressed_info(h)[1] for h in hs)
        dec, link = zf.zf_ctx_rates(g.ctx, zf.ZF_DELTA_BP, zf.ZF_I64, 8)
        assert dec == 0.0 and link == pytest.approx(comp / (ms * 1e6), rel=1e-3) and link > 1.0
        (x, s, cr), h = cols[0], hs[0]
        buf = g.alloc(out_specs(x))[0]
        pts, best = zf.zf_tune(g.ctx, [h], [buf.data_ptr()], [buf.numel()], transfer=False, reps=2)
        raw = zf.zf_compressed_info(h)[0]
        rates = [zf.zf_ctx_rates(g.ctx, zf.ZF_DELTA_BP, zf.ZF_I64, w)[0] for w in (8, 16, 32, 64)]
        assert any(r == pytest.approx(raw / (min(p.ms for p in pts) * 1e6), rel=1e-3) for r in rates)
        specs = [sp for x2, s2, cr2 in cols for sp in out_specs(x2)]
        for flags, order in ((0, [0, 1, 2]), (zf.ZF_KCFG_KEEP_ORDER, [0, 1, 2]), (zf.ZF_KCFG_KEEP_ORDER, [2, 1, 0])):
            zf.zf_ctx_set_kcfg(g.ctx, 0, 0, 0, 1 << 20, flags)
            got = g.decode([hs[i] for i in order], [specs[i] for i in order])
            for i, y in zip(order, got):
                assert np.array_equal(y, cols[i][0]), (flags, order)
    finally:
        g.close()


def test_tune_chunk_rows_times_every_candidate(columns):
    """The chunk-size dimension of the search: every candidate chunk size is
    encoded and timed through the transfer, one that does not fit (not a
    multiple of 1024 rows) gets -1, the fastest is reported, and the column
    encoded at that size decodes exactly."""
    cols, hs = columns
    (x, s, cr) = cols[1]                                   # the RLE dates
    g = Gpu()
    try:
        cand = [65536, 262144, 1000, 1 << 20]
        ms, best = zf.zf_tune_chunk_rows(g.ctx, zf.Column(x), s, cand, reps=2)
        assert ms[2] == -1.0 and all(ms[i] > 0 for i in (0, 1, 3))
        assert best in (0, 1, 3) and ms[best] == min(ms[i] for i in (0, 1, 3))
        h = compress(x, s, cand[best])
        try:
            got, = g.decode([h], out_specs(x))
            assert np.array_equal(got, x)
        finally:
            zf.zf_compressed_free(h)
    finally:
        g.close()
