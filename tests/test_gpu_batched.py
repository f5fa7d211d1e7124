"""The batched workload at full size: a 16-column, 400M-row fact table
(40 GB uncompressed) streamed in ~1,800 uneven 4-64 MB pieces through one
call -- one work-queue launch per stage, captured in a CUDA graph and
replayed -- checked column by column against the generated data, and on
sampled pieces against the oracle's own decode."""
import numpy as np
import pytest

import oracle
import zf_workloads as W

zf = pytest.importorskip("paper_2602_08190_gb300")
pytestmark = pytest.mark.gpu


def test_fact_table_40gb_batched_graph():
    import torch
    import bench
    cfg = bench.build_c4(zf, 1, bench.FACT_ROWS, keep=True)
    cols = cfg.expects
    handles = cfg.handles
    try:
        raw = sum(c.nbytes for c in cols)
        assert raw == 40_000_000_000
        ctx = zf.zf_ctx_create(0)
        zf.zf_ctx_set_kcfg(ctx, 0, 0, 0, 64 << 20, zf.ZF_KCFG_BATCHED | zf.ZF_KCFG_GRAPH)
        zf.zf_ctx_set_ring(ctx, 3)
        dev = [torch.empty(c.nbytes, dtype=torch.uint8, device="cuda") for c in cols]
        outs, caps = [], []
        for parts in cfg.parts:
            for ci, off, n in parts:
                outs.append(dev[ci].data_ptr() + off)
                caps.append(n)
        for rep in range(2):                       # capture, then replay
            for d in dev:
                d.fill_(0x5A)
            torch.cuda.synchronize()               # the library runs on its own streams
            zf.zf_transfer_decompress(ctx, handles, outs, caps)
            st, stats = zf.zf_sync(ctx)
            assert stats.raw_bytes == raw and stats.n_chunks == len(handles)
            for ci, c in enumerate(cols):
                assert np.array_equal(dev[ci].cpu().numpy().view(c.dtype), c), (rep, W.FACT_COLUMNS[ci][0])
        # sampled pieces decoded by the oracle from the library's bytes
        rng = np.random.default_rng(4)
        for k in rng.choice(len(handles), 16, replace=False):
            (ci, off, n), = cfg.parts[k]
            isz = cols[ci].itemsize
            ref = oracle.decode(zf.zf_compressed_bytes(handles[k]))
            assert np.array_equal(ref, cols[ci][off // isz:(off + n) // isz])
        zf.zf_ctx_destroy(ctx)
    finally:
        cfg.free(zf)
